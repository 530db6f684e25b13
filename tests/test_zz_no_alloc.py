"""The no-allocation pointwise estimator.

Some callers cannot allocate device memory: code running inside a framework
whose allocator owns every byte of the GPU, host callbacks in which CUDA
allocation calls are not allowed, or tight loops that cannot pay for the
device-wide synchronisation of cudaMalloc/cudaFree.  For them the library
offers wos_estimate_static_scratch, which runs the pointwise walk-on-spheres
estimator with a static 16 MiB device array inside the library as its
scratch.  This test calls it through the C ABI and checks, on two calls in a
row (the second reuses the array with the previous call's contents still in
it), that it gives what the workspace-based wos_estimate gives.

The file is named so that pytest collects it last.
"""
import ctypes as C

import numpy as np
import pytest
import torch

from paper_2302_11825_gb300 import bvc
from paper_2302_11825_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def test_static_scratch_estimator_matches_workspace_estimator():
    w = wl.star_poisson(n_samples=16, walks=4, grid=96, n_seg=4000, manufactured=True)
    geom = bvc.Geometry(w.V, w.F)
    near = bvc.classify_near(geom, bvc.soa(w.eval_pts), w.offset_l).cpu().numpy().astype(bool)
    pts = bvc.soa(w.eval_pts[~near][:3000])
    walks = 512  # 6 KB of records per point: 3000 points need two passes through the 16 MiB array
    eps, max_steps, seed = w.eps, 1 << 14, 21
    lib = bvc.lib()
    g, f = bvc.make_function(w.g), bvc.make_function(w.f)
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    a = bvc.EvalState(pts)   # filled by the no-allocation entry point
    b = bvc.EvalState(pts)   # filled by wos_estimate with its own workspace
    m = pts.shape[1]
    for call in range(2):
        id_base = call * m * walks
        st = lib.wos_estimate_static_scratch(geom.h, C.byref(g), C.byref(f), C.byref(a.struct), walks, eps,
                                             max_steps, seed, id_base, stream)
        assert st == bvc.OK, bvc.status_string(st)
        bvc.wos_estimate(geom, w.g, w.f, b, walks, eps, max_steps, seed, id_base)
        torch.cuda.synchronize()
        assert a.counts.cpu().tolist() == b.counts.cpu().tolist() == [(call + 1) * walks, 0]
        np.testing.assert_allclose(a.u_bnd.cpu().numpy(), b.u_bnd.cpu().numpy(), rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(a.grad_bnd.cpu().numpy(), b.grad_bnd.cpu().numpy(), rtol=1e-12, atol=1e-12)
    ua, _ = bvc.get_solution(a)
    assert np.all(np.isfinite(ua.cpu().numpy()))
    # one point's records must fit in the array: beyond that the call is refused
    st = lib.wos_estimate_static_scratch(geom.h, C.byref(g), C.byref(f), C.byref(a.struct), 1_400_000, eps,
                                         max_steps, seed, 0, stream)
    assert st == bvc.ERR_WORKSPACE
