"""The debug build (libbvc_debug.so, compiled with BVC_DEBUG=1): bounds checks
in every device BVH traversal that set a status flag and skip the access
instead of faulting.

Each case runs in a child process whose first library load picks the debug
build (environment BVC_DEBUG=1).  On intact trees the debug build gives
results identical to the release build's (loaded by this process) and sets
no flag.  With one child link of the device tree overwritten -- a node index
past the tree, or a leaf whose primitive range runs past the primitive
count -- the walks still finish and bvc_geometry_stats returns
BVC_ERR_BOUNDS with bit 1 of the flags set.  The overwritten links are out
of range only, never an in-range index (which could close a cycle that no
range check sees), so every access of a corrupted run is checked before it
is made."""
import os
import subprocess
import sys

import numpy as np
import pytest
import torch

from paper_2302_11825_gb300 import bvc
from paper_2302_11825_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
MAX_STEPS = 256  # bounds the walks of a corrupted tree, which may leave the domain


def _cases():
    return {
        2: wl.circle_laplace(n_samples=1024, walks=8, grid=24),
        3: wl.icosphere_laplace(subdiv=3, n_samples=1024, walks=8, plane=16, n_random=400),
    }


def _run(w, geom, seed=3):
    """One cache build, an evaluation and a closest-point query."""
    opts = bvc.cache_opts(w.n_samples, w.walks, w.offset_l, w.eps, seed, max_steps=MAX_STEPS)
    cache = bvc.cache_build(geom, w.g, w.f, opts, bvc.Cache(w.dim, w.n_samples))
    st = bvc.EvalState(bvc.soa(w.eval_pts), grad=False)
    bvc.evaluate(cache, st)
    u, _ = bvc.get_solution(st)
    d2, prim, _ = bvc.query_closest(geom, bvc.soa(w.eval_pts))
    torch.cuda.synchronize()
    return {"u_hat": cache.u_hat.cpu().numpy(), "q_hat": cache.dudn_hat.cpu().numpy(), "u": u.cpu().numpy(),
            "d2": d2.cpu().numpy(), "prim": prim.cpu().numpy()}


def _child(out_path):
    """Runs in the debug child: intact results, then two corrupted trees."""
    assert bvc.debug_build(), "BVC_DEBUG=1 did not load the debug build"
    res = {}
    for dim, w in _cases().items():
        geom = bvc.Geometry(w.V, w.F)
        intact = _run(w, geom)
        s = geom.stats(reset=True)
        res[f"{dim}_intact_status"] = s["status"]
        res[f"{dim}_intact_flags"] = s["flags"]
        for k, v in intact.items():
            res[f"{dim}_{k}"] = v
        info = geom.info()
        # the root's right child: a node index past the tree
        geom.debug_set_link(0, 1, int(info.n_nodes) + 1000)
        _run(w, geom)
        s = geom.stats(reset=True)
        res[f"{dim}_node_status"], res[f"{dim}_node_flags"] = s["status"], s["flags"]
        # a fresh tree, the root's left child: a leaf past the primitives
        geom2 = bvc.Geometry(w.V, w.F)
        geom2.debug_set_link(0, 0, ~(((int(info.n_prims) + 16) << 4) | 3))
        _run(w, geom2)
        s = geom2.stats(reset=True)
        res[f"{dim}_leaf_status"], res[f"{dim}_leaf_flags"] = s["status"], s["flags"]
    np.savez(out_path, **res)


def test_debug_build_checks_bounds(work_dir):
    out = os.path.join(work_dir, "debug.npz")
    env = dict(os.environ, BVC_DEBUG="1", PYTHONPATH=ROOT + os.pathsep + os.environ.get("PYTHONPATH", ""))
    r = subprocess.run([sys.executable, os.path.abspath(__file__), out], env=env, cwd=ROOT, capture_output=True,
                       text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    got = np.load(out)
    assert not bvc.debug_build()
    for dim, w in _cases().items():
        ref = _run(w, bvc.Geometry(w.V, w.F))
        # no flag on an intact tree; the debug build's results are the release build's
        assert got[f"{dim}_intact_status"] in (bvc.OK, bvc.WARN_WALK_CAP) and got[f"{dim}_intact_flags"] == 0
        for k, v in ref.items():
            assert np.array_equal(got[f"{dim}_{k}"], v, equal_nan=True), (dim, k)
        for case in ("node", "leaf"):
            assert got[f"{dim}_{case}_status"] == bvc.ERR_BOUNDS, (dim, case, int(got[f"{dim}_{case}_status"]))
            assert int(got[f"{dim}_{case}_flags"]) & 2, (dim, case)
        print(f"[debug build {dim}D] intact results identical to the release build; "
              f"corrupted node and leaf links reported as BVC_ERR_BOUNDS")


def test_release_build_refuses_the_link_hook():
    w = wl.circle_laplace(n_samples=64, walks=2, grid=8)
    geom = bvc.Geometry(w.V, w.F)
    st = bvc.lib().bvc_debug_set_link(geom.h, 0, 1, 7, None)
    assert st == bvc.ERR_UNSUPPORTED
    assert bvc.lib().bvc_debug_set_link(geom.h, int(geom.info().n_nodes), 0, 7, None) == bvc.ERR_INVALID_ARG
    assert bvc.lib().bvc_debug_set_link(geom.h, 0, 2, 7, None) == bvc.ERR_INVALID_ARG


if __name__ == "__main__":
    _child(sys.argv[1])
