"""The walk autotuner: it picks a launch shape within the documented range
and, because a walk's result depends only on its id, caches built with any
shape are identical bit for bit."""
import pytest
import torch

from paper_2302_11825_gb300 import bvc
from paper_2302_11825_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def test_tuned_and_forced_shapes_give_identical_caches():
    w = wl.star_poisson(n_samples=4096, walks=32, grid=16, n_seg=4000, src_grid=(32, 32))
    geom = bvc.Geometry(w.V, w.F)
    opts = bvc.cache_opts(w.n_samples, w.walks, w.offset_l, w.eps, 5, src_grid=(32, 32))
    ref = bvc.cache_build(geom, w.g, w.f, opts, bvc.Cache(2, w.n_samples, n_src_cand=32 * 32))
    b, c, ms = bvc.tune_walks(geom, w.g, w.f, opts)
    print(f"[tune] blocks/SM={b} chunk={c} best={ms:.3f} ms")
    assert b >= 1 and c in (64, 128, 256) and ms > 0
    tuned = bvc.cache_build(geom, w.g, w.f, opts, bvc.Cache(2, w.n_samples, n_src_cand=32 * 32))
    bvc.set_walk_shape(geom, 2, 32)
    forced = bvc.cache_build(geom, w.g, w.f, opts, bvc.Cache(2, w.n_samples, n_src_cand=32 * 32))
    torch.cuda.synchronize()
    for x in (tuned, forced):
        assert torch.equal(x.u_hat, ref.u_hat) and torch.equal(x.dudn_hat, ref.dudn_hat)
    bvc.set_walk_shape(geom, 0, 0)
