"""Host code under AddressSanitizer and UBSan (CPU): the BVH builder the
library uploads (structure checked by tests/host/bvh_check.cpp on meshes of
the workloads and on degenerate inputs -- coincident elements, one or two
elements), and the C oracle's main entry points (tests/host/oracle_check.c)."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from paper_2302_11825_gb300 import workloads as wl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SAN = ["-O1", "-g", "-fsanitize=address,undefined", "-fno-sanitize-recover=undefined", "-fno-omit-frame-pointer"]


def _cuda_include():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.realpath(nvcc))), "include")
    return inc if os.path.exists(os.path.join(inc, "vector_types.h")) else None


def _compile(cmd):
    if shutil.which(cmd[0]) is None:
        pytest.skip(f"{cmd[0]} not found")
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0 and "sanitize" in r.stderr and "cannot find" in r.stderr:
        pytest.skip("sanitizer runtime not installed")
    assert r.returncode == 0, r.stderr[-3000:]


def _write_mesh(path, V, F):
    V = np.ascontiguousarray(V, np.float32)
    F = np.ascontiguousarray(F, np.int32)
    with open(path, "wb") as f:
        f.write(np.int32(V.shape[1]).tobytes())
        f.write(np.int64(V.shape[0]).tobytes())
        f.write(np.int64(F.shape[0]).tobytes())
        f.write(V.tobytes())
        f.write(F.tobytes())


def _meshes():
    out = {"circle256": wl.circle_polygon(256), "star20k": wl.star_polygon(20000, 0)}
    out["icosphere4"] = wl.icosphere(4)
    out["channel"] = wl.box_with_obstacles(n_box=4, ellipsoids=[((0.0, 0.0, 0.0), (0.5, 0.35, 0.35))], subdiv=3)
    seg = np.array([[0.0, 0.0], [1.0, 0.5]], np.float32)
    out["coincident2d"] = (seg, np.tile(np.array([[0, 1]], np.int32), (600, 1)))
    tri = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.0, 1.0, 0.2]], np.float32)
    out["coincident3d"] = (tri, np.tile(np.array([[0, 1, 2]], np.int32), (300, 1)))
    out["one2d"] = (seg, np.array([[0, 1]], np.int32))
    out["two3d"] = (np.concatenate([tri, tri + 1.0]), np.array([[0, 1, 2], [3, 4, 5]], np.int32))
    return out


def test_bvh_builder_structure_under_sanitizers(work_dir):
    inc = _cuda_include()
    if inc is None:
        pytest.skip("CUDA headers (vector_types.h) not found")
    exe = os.path.join(work_dir, "bvh_check")
    _compile(["g++", "-std=c++17", *SAN, "-I", inc, os.path.join(ROOT, "tests", "host", "bvh_check.cpp"),
              os.path.join(ROOT, "paper_2302_11825_gb300", "csrc", "bvh_build.cpp"), "-o", exe])
    for name, (V, F) in _meshes().items():
        path = os.path.join(work_dir, name + ".bin")
        _write_mesh(path, V, F)
        r = subprocess.run([exe, path], capture_output=True, text=True, timeout=300)
        assert r.returncode == 0 and "ERROR" not in r.stderr and "runtime error" not in r.stderr, \
            (name, r.stdout, r.stderr[-3000:])


def _write_problem(path, V, F, neu, g_terms, pts):
    import oracle
    V = np.ascontiguousarray(V, np.float32)
    F = np.ascontiguousarray(F, np.int32)
    g = np.ascontiguousarray(oracle.encode_function(g_terms), np.float64)
    pts = np.ascontiguousarray(pts, np.float64)
    with open(path, "wb") as f:
        f.write(np.int32(V.shape[1]).tobytes())
        f.write(np.int64(V.shape[0]).tobytes())
        f.write(np.int64(F.shape[0]).tobytes())
        f.write(V.tobytes())
        f.write(F.tobytes())
        f.write(np.ascontiguousarray(neu, np.uint8).tobytes())
        f.write(np.int64(g.size).tobytes())
        f.write(g.tobytes())
        f.write(np.int64(pts.shape[0]).tobytes())
        f.write(pts.tobytes())


def test_oracle_under_sanitizers(work_dir):
    exe = os.path.join(work_dir, "oracle_check")
    _compile(["gcc", "-std=c11", *SAN, "-fopenmp", "-ffp-contract=off",
              os.path.join(ROOT, "tests", "host", "oracle_check.c"), os.path.join(ROOT, "oracle", "bvc_oracle.c"),
              "-o", exe, "-lm"])
    V2, F2 = wl.l_shape_polygon(8)
    mid = wl.element_midpoints(V2, F2)
    neu2 = (mid[:, 0] > -1 + 1e-6).astype(np.uint8)
    rng = np.random.default_rng(1)
    p2 = rng.uniform(-0.9, 0.9, (200, 2))
    p2 = p2[~((p2[:, 0] > 0) & (p2[:, 1] > 0))][:64]
    b = wl.box_mixed_3d()
    p3 = rng.uniform(0.1, 0.9, (64, 3))
    cases = {"lshape": (V2, F2, neu2, [(wl.POLY, wl.poly2d_coeffs({(2, 0): 1.0, (0, 2): -1.0}))], p2),
             "cube": (b.V, b.F, b.neumann, b.g, p3)}
    env = dict(os.environ, OMP_NUM_THREADS="2", ASAN_OPTIONS="detect_leaks=1")
    for name, (V, F, neu, g, p) in cases.items():
        path = os.path.join(work_dir, name + ".bin")
        _write_problem(path, V, F, neu, g, p)
        r = subprocess.run([exe, path], capture_output=True, text=True, timeout=600, env=env)
        assert r.returncode == 0 and "ERROR" not in r.stderr and "runtime error" not in r.stderr, \
            (name, r.stdout, r.stderr[-3000:])
