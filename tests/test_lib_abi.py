"""The C-ABI library builds, loads and exports every entry point that
include/bvc.h declares; host-side argument validation needs no GPU; the
product package never touches the oracle."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "bvc.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b((?:bvc|wost?)_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2302_11825_gb300 import build
    path = build.build()
    return C.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared()
    for required in ["bvc_geometry_create", "bvc_cache_build", "bvc_evaluate", "wos_estimate",
                     "bvc_query_closest", "bvc_walk", "bvc_sample_boundary", "bvc_get_solution"]:
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_host_only_calls(lib):
    lib.bvc_version.restype = C.c_int32
    assert lib.bvc_version() >= 100
    lib.bvc_status_string.restype = C.c_char_p
    lib.bvc_status_string.argtypes = [C.c_int]
    assert lib.bvc_status_string(0) == b"ok"
    assert b"workspace" in lib.bvc_status_string(7)
    assert b"bounds" in lib.bvc_status_string(9)
    # the release build: no device bounds checks, the link hook refused
    lib.bvc_debug_build.restype = C.c_int32
    assert lib.bvc_debug_build() == 0
    lib.bvc_debug_set_link.restype = C.c_int
    lib.bvc_debug_set_link.argtypes = [C.c_void_p, C.c_int64, C.c_int32, C.c_int32, C.c_void_p]
    assert lib.bvc_debug_set_link(None, 0, 0, 0, None) == 1  # BVC_ERR_INVALID_ARG


def _create(lib, V, F):
    lib.bvc_geometry_create.restype = C.c_int
    lib.bvc_geometry_create.argtypes = [C.c_int32, C.c_void_p, C.c_int64, C.c_void_p, C.c_int64, C.c_void_p,
                                        C.POINTER(C.c_void_p)]
    h = C.c_void_p()
    V = np.ascontiguousarray(V, np.float32)
    F = np.ascontiguousarray(F, np.int32)
    st = lib.bvc_geometry_create(V.shape[1], V.ctypes.data_as(C.c_void_p), V.shape[0],
                                 F.ctypes.data_as(C.c_void_p), F.shape[0], None, C.byref(h))
    return st, h


def test_geometry_validation_on_host(lib):
    # every rejection below happens before any CUDA call
    V = np.array([[0, 0], [1, 0], [0, 1]], np.float32)
    F = np.array([[0, 1], [1, 2], [2, 0]], np.int32)
    bad_v = V.copy()
    bad_v[1, 0] = np.nan
    assert _create(lib, bad_v, F)[0] == 2          # non-finite vertex
    assert _create(lib, V, np.array([[0, 1], [1, 5], [2, 0]]))[0] == 2  # index out of range
    assert _create(lib, V, np.array([[0, 1], [1, 1], [2, 0]]))[0] == 2  # zero-length segment
    tri = np.array([[0, 0, 0], [1, 0, 0], [2, 0, 0]], np.float32)
    assert _create(lib, tri, np.array([[0, 1, 2]]))[0] == 2             # zero-area triangle
    lib.bvc_geometry_create.argtypes = [C.c_int32, C.c_void_p, C.c_int64, C.c_void_p, C.c_int64, C.c_void_p,
                                        C.POINTER(C.c_void_p)]
    h = C.c_void_p()
    assert lib.bvc_geometry_create(4, None, 3, None, 3, None, C.byref(h)) == 1
    assert lib.bvc_geometry_create(2, None, 3, None, 3, None, None) == 1


def test_entry_points_reject_null_handles(lib):
    lib.bvc_query_closest.restype = C.c_int
    assert lib.bvc_query_closest(None, None, C.c_int64(4), None, None, None, None) == 1
    lib.bvc_walk.restype = C.c_int
    assert lib.bvc_walk(None, None, None, None, None, C.c_int64(1), C.c_int32(1), C.c_float(1e-3), C.c_int32(10),
                        C.c_uint64(0), C.c_uint64(0), C.c_uint32(0), None, None, None, None) == 1
    lib.bvc_cache_build.restype = C.c_int
    assert lib.bvc_cache_build(None, None, None, None, None, None, C.c_size_t(0), None) == 1
    lib.bvc_evaluate.restype = C.c_int
    assert lib.bvc_evaluate(None, None, None, C.c_size_t(0), None) == 1
    lib.wos_estimate.restype = C.c_int
    assert lib.wos_estimate(None, None, None, None, C.c_int64(1), C.c_int32(1), C.c_float(1e-3), C.c_int32(1),
                            C.c_uint64(0), C.c_uint64(0), None, None, None, C.c_size_t(0), None) == 1


def test_debug_build_is_a_separate_library(work_dir):
    # the debug variant compiles (BVC_DEBUG=1) and says so; the release
    # library is left as it was
    from paper_2302_11825_gb300 import build
    path = build.build(debug=True)
    assert path.endswith("libbvc_debug.so") and path != build.LIB
    dbg = C.CDLL(path)
    dbg.bvc_debug_build.restype = C.c_int32
    assert dbg.bvc_debug_build() == 1
    missing = [n for n in _declared() if not hasattr(dbg, n)]
    assert not missing, missing


def test_last_error_is_thread_local_and_cleared(lib):
    import threading
    lib.bvc_last_error.restype = C.c_int
    lib.bvc_last_error()  # start clean
    lib.bvc_query_closest.restype = C.c_int
    assert lib.bvc_query_closest(None, None, C.c_int64(4), None, None, None, None) == 1
    seen = []
    t = threading.Thread(target=lambda: seen.append(lib.bvc_last_error()))
    t.start()
    t.join()
    assert seen == [0]                   # another thread saw no error
    assert lib.bvc_last_error() == 1     # this thread's last error (invalid argument) ...
    assert lib.bvc_last_error() == 0     # ... cleared by the read
    mn, full = C.c_size_t(), C.c_size_t()
    lib.wos_estimate_workspace_size.restype = C.c_int
    assert lib.wos_estimate_workspace_size(2, C.c_int64(10), 4, C.byref(mn), C.byref(full)) == 0
    assert lib.bvc_last_error() == 0     # successful calls leave it alone


def test_gather_shape_host_checks(lib):
    lib.bvc_set_gather_shape.restype = C.c_int
    assert lib.bvc_set_gather_shape(2, 0, 5) == 1 and lib.bvc_set_gather_shape(4, 0, 4) == 1
    assert lib.bvc_set_gather_shape(3, 1, 6) == 1 and lib.bvc_set_gather_shape(3, 2, 4) == 1
    assert lib.bvc_set_gather_shape(3, 0, 4) == 0 and lib.bvc_set_gather_shape(3, 0, 0) == 0
    lib.bvc_tune_gather.restype = C.c_int
    assert lib.bvc_tune_gather(None, None, None, C.c_size_t(0), None, None, None) == 1


def test_workspace_size_queries_are_host_only(lib):
    lib.wos_estimate_workspace_size.restype = C.c_int
    mn, full = C.c_size_t(), C.c_size_t()
    assert lib.wos_estimate_workspace_size(2, C.c_int64(1000), 64, C.byref(mn), C.byref(full)) == 0
    per_point = 64 * 3 * 4 + 4 * 4  # walk records + the shared first closest-point hit
    assert full.value == 512 + 1000 * per_point and mn.value == 512 + per_point
    lib.bvc_sample_source_workspace_size.restype = C.c_int
    b = C.c_size_t()
    assert lib.bvc_sample_source_workspace_size(C.c_int64(65536), C.byref(b)) == 0 and b.value > 65536 * 8


def test_product_does_not_use_the_oracle():
    pkg = os.path.join(ROOT, "paper_2302_11825_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".cpp", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "liboracle" not in text and "bvc_oracle" not in text, f


def test_missing_library_fails_loudly(monkeypatch):
    """Without the CUDA library (and no way to build it) every call raises:
    there is no CPU fallback."""
    from paper_2302_11825_gb300 import bvc
    from paper_2302_11825_gb300 import build as b

    def no_toolkit(*a, **k):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libbvc.so")

    monkeypatch.setattr(bvc, "_lib", None)
    monkeypatch.setattr(b, "LIB", os.path.join(ROOT, "tests", "_tmp", "missing", "libbvc.so"))
    monkeypatch.setattr(b, "build", no_toolkit)
    with pytest.raises(RuntimeError, match="CUDA toolkit"):
        bvc.lib()
    V = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0]], np.float32)
    F = np.array([[0, 1], [1, 2], [2, 0]], np.int32)
    with pytest.raises(RuntimeError, match="CUDA toolkit"):
        bvc.Geometry(V, F)


def test_device_allocation_failure_is_an_error(lib):
    """On a machine without a GPU every device allocation fails: the creating
    calls return an error and leave the handle NULL (no crash, no leak of a
    half-built handle)."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present: allocations succeed")
    from paper_2302_11825_gb300 import workloads as wl
    V, F = wl.circle_polygon(64)
    V = np.ascontiguousarray(V, np.float32)
    F = np.ascontiguousarray(F, np.int32)
    vp, fp = V.ctypes.data_as(C.c_void_p), F.ctypes.data_as(C.c_void_p)
    lib.bvc_geometry_create.restype = C.c_int
    lib.bvc_geometry_create.argtypes = [C.c_int32, C.c_void_p, C.c_int64, C.c_void_p, C.c_int64, C.c_void_p,
                                        C.POINTER(C.c_void_p)]
    h = C.c_void_p(1)
    st = lib.bvc_geometry_create(2, vp, V.shape[0], fp, F.shape[0], None, C.byref(h))
    assert st not in (0, 1) and h.value is None
    lib.bvc_mixed_create.restype = C.c_int
    lib.bvc_mixed_create.argtypes = [C.c_int32, C.c_void_p, C.c_int64, C.c_void_p, C.c_int64, C.c_void_p,
                                     C.c_void_p, C.POINTER(C.c_void_p)]
    neu = np.zeros(F.shape[0], np.uint8)
    neu[:10] = 1
    h = C.c_void_p(1)
    st = lib.bvc_mixed_create(2, vp, V.shape[0], fp, F.shape[0], neu.ctypes.data_as(C.c_void_p), None, C.byref(h))
    assert st not in (0, 1) and h.value is None


def test_multi_rhs_host_checks(lib):
    lib.bvc_poly_terms.restype = C.c_int32
    assert [lib.bvc_poly_terms(d) for d in (1, 2, 3, 4)] == [0, 15, 35, 0]
    lib.bvc_multi_cache_build_workspace_size.restype = C.c_int
    mn = C.c_size_t()
    assert lib.bvc_multi_cache_build_workspace_size(None, C.c_int64(10), 4, C.byref(mn), None) == 1
    lib.bvc_multi_cache_build.restype = C.c_int
    assert lib.bvc_multi_cache_build(None, None, None, None, None, C.c_size_t(0), None) == 1
    lib.bvc_multi_cache_project.restype = C.c_int
    assert lib.bvc_multi_cache_project(None, None, None) == 1
    lib.bvc_evaluate_multi.restype = C.c_int
    assert lib.bvc_evaluate_multi(None, None, C.c_int64(0), None, None) == 1
    # the source variant: null handles and arguments are argument errors
    lib.bvc_multi_cache_build_source_workspace_size.restype = C.c_int
    assert lib.bvc_multi_cache_build_source_workspace_size(None, None, C.byref(mn), None) == 1
    lib.bvc_multi_cache_build_source.restype = C.c_int
    assert lib.bvc_multi_cache_build_source(None, None, None, None, None, None, C.c_size_t(0), None) == 1


def test_harmonic_polynomial_generator():
    # the random right-hand sides of the batched workload are harmonic:
    # the Laplacian of each, by central differences, vanishes
    from paper_2302_11825_gb300 import workloads as wl
    for dim, nb in ((2, 9), (3, 25)):
        assert wl.harmonic_basis(dim).shape == (nb, 15 if dim == 2 else 35)
        C = wl.random_harmonic_polys(dim, 4, seed=1)
        x = np.random.default_rng(2).uniform(-1, 1, (50, dim))
        h = 1e-3
        for k in range(4):
            t = [(wl.POLY, C[k])]
            f0 = wl.eval_terms(t, dim, x)[0]
            lap = sum(wl.eval_terms(t, dim, x + h * e)[0] + wl.eval_terms(t, dim, x - h * e)[0] - 2 * f0
                      for e in np.eye(dim)) / h ** 2
            assert np.abs(lap).max() < 1e-4 * max(1.0, np.abs(f0).max())


def test_batch_host_checks(lib):
    lib.bvc_batch_create.restype = C.c_int
    h = C.c_void_p()
    assert lib.bvc_batch_create(None, 1, 4, 10, 1, None, C.byref(h)) == 1
    assert lib.bvc_batch_create(None, 0, 4, 10, 1, None, None) == 1
    for name, nargs in (("bvc_batch_destroy", 1), ("bvc_batch_get_info", 4), ("bvc_batch_build_workspace_size", 3),
                        ("bvc_batch_build", 7), ("bvc_batch_project", 4), ("bvc_batch_evaluate", 5),
                        ("bvc_batch_set_counting", 2), ("bvc_batch_stats", 4)):
        fn = getattr(lib, name)
        fn.restype = C.c_int
        args = [None] * nargs
        if name == "bvc_batch_build":
            args = [None, None, None, None, None, C.c_size_t(0), None]
        assert fn(*args) == 1, name


def test_region_clamp_screened_host_checks(lib):
    lib.bvc_cache_build_region.restype = C.c_int
    assert lib.bvc_cache_build_region(None, None, None, None, None, None, None, C.c_size_t(0), None) == 1
    lib.bvc_clamp_correction_workspace_size.restype = C.c_int
    b = C.c_size_t()
    assert lib.bvc_clamp_correction_workspace_size(2, C.c_int64(100), 4, 8, C.byref(b)) == 0 and b.value > 0
    assert lib.bvc_clamp_correction_workspace_size(4, C.c_int64(100), 4, 8, C.byref(b)) == 1
    lib.bvc_clamp_correction.restype = C.c_int
    assert lib.bvc_clamp_correction(None, None, C.c_double(0.0), None, None, C.c_double(0.0), C.c_double(1.0), None,
                                    C.c_int64(0), 1, 1, C.c_float(1e-3), 10, C.c_uint64(0), None, None, None,
                                    C.c_size_t(0), None) == 1
    lib.wos_estimate_sigma.restype = C.c_int
    assert lib.wos_estimate_sigma(None, None, None, C.c_double(1.0), None, 1, C.c_float(1e-3), 10, C.c_uint64(0),
                                  C.c_uint64(0), None, C.c_size_t(0), None) == 1
    lib.bvc_tune_walks_workspace_size.restype = C.c_int
    assert lib.bvc_tune_walks_workspace_size(None, None, None) == 1


def test_mixed_host_checks(lib):
    """Mixed boundaries: argument errors are caught on the host, before any
    device work (no GPU needed)."""
    lib.bvc_mixed_create.restype = C.c_int
    lib.bvc_mixed_create.argtypes = [C.c_int32, C.c_void_p, C.c_int64, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p,
                                     C.POINTER(C.c_void_p)]
    from paper_2302_11825_gb300 import workloads as wl
    V, F, side = wl.rect_polygon((0, 0), (1, 1), 4)
    V = np.ascontiguousarray(V, np.float32)
    F = np.ascontiguousarray(F, np.int32)
    h = C.c_void_p()
    all_neu = np.ones(F.shape[0], np.uint8)
    vp, fp = V.ctypes.data_as(C.c_void_p), F.ctypes.data_as(C.c_void_p)
    # no Dirichlet element: walks could never stop
    assert lib.bvc_mixed_create(2, vp, V.shape[0], fp, F.shape[0], all_neu.ctypes.data_as(C.c_void_p), None,
                                C.byref(h)) == 1
    assert lib.bvc_mixed_create(4, vp, V.shape[0], fp, F.shape[0], all_neu.ctypes.data_as(C.c_void_p), None,
                                C.byref(h)) == 1
    assert lib.bvc_mixed_create(2, vp, V.shape[0], fp, F.shape[0], None, None, C.byref(h)) == 1
    assert lib.bvc_mixed_create(2, vp, V.shape[0], fp, F.shape[0], None, None, None) == 1
    for name in ("bvc_mixed_destroy", "bvc_mixed_get_info"):
        fn = getattr(lib, name)
        fn.restype = C.c_int
    lib.bvc_mixed_destroy.argtypes = [C.c_void_p]
    assert lib.bvc_mixed_destroy(None) == 1
    lib.bvc_mixed_cache_build_workspace_size.restype = C.c_int
    lib.bvc_mixed_cache_build_workspace_size.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
    assert lib.bvc_mixed_cache_build_workspace_size(None, None, None, None) == 1
    lib.wost_estimate.restype = C.c_int
    lib.wost_estimate.argtypes = [C.c_void_p] * 5 + [C.c_int32, C.c_float, C.c_int32, C.c_uint64, C.c_uint64,
                                                      C.c_void_p, C.c_size_t, C.c_void_p]
    assert lib.wost_estimate(None, None, None, None, None, 1, 1e-3, 10, 0, 0, None, 0, None) == 1
    lib.bvc_mixed_set_silhouette_gap.restype = C.c_int
    lib.bvc_mixed_set_silhouette_gap.argtypes = [C.c_void_p, C.c_double]
    assert lib.bvc_mixed_set_silhouette_gap(None, 0.1) == 1


def test_wait_selftest_rejects_bad_limits(lib):
    lib.bvc_wait_selftest.restype = C.c_int
    lib.bvc_wait_selftest.argtypes = [C.c_int64, C.c_void_p]
    assert lib.bvc_wait_selftest(-1, None) == 1
    assert lib.bvc_wait_selftest(3_000_000_000, None) == 1


def test_header_is_plain_c_and_links(work_dir):
    """include/bvc.h compiles as C11 with -pedantic -Werror, and a C program
    linked against the library gets the declared host-side behaviour."""
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("gcc not found")
    from paper_2302_11825_gb300 import build as b
    lib_path = b.build()
    exe = os.path.join(work_dir, "abi_c_check")
    r = subprocess.run(["gcc", "-std=c11", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I",
                        os.path.join(ROOT, "include"), os.path.join(ROOT, "tests", "host", "abi_c_check.c"),
                        "-o", exe, lib_path, "-Wl,-rpath," + os.path.dirname(lib_path)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-3000:]
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, (r.stdout, r.stderr[-2000:])
