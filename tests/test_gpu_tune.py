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


@pytest.mark.parametrize("dim", [2, 3])
def test_gather_tuner_picks_a_supported_shape_with_the_same_results(dim):
    # every points-per-thread count accumulates each point's pairs in the
    # same order within a tile; the split of the samples across CTAs (and so
    # the FP64 grouping) may differ, so results agree to FP64 rounding
    if dim == 2:
        w = wl.star_poisson(n_samples=4096, walks=16, grid=64, n_seg=4000, src_grid=(48, 48))
        src = (48, 48)
    else:
        w = wl.icosphere_laplace(subdiv=4, n_samples=4096, walks=16, plane=32, n_random=3000)
        src = (0, 0)
    geom = bvc.Geometry(w.V, w.F)
    n_src = bvc.n_candidates(dim, src) if src[0] else 0
    opts = bvc.cache_opts(w.n_samples, w.walks, w.offset_l, w.eps, 5, src_grid=src)
    cache = bvc.cache_build(geom, w.g, w.f, opts, bvc.Cache(dim, w.n_samples, n_src_cand=n_src))
    st = bvc.EvalState(bvc.soa(w.eval_pts))
    outs = []
    for pts in (2, 4, 6):
        bvc.set_gather_shape(dim, 0, pts)
        bvc.set_gather_shape(dim, 1, 4 if pts == 4 else 2)
        bvc.eval_state_reset(st)
        bvc.evaluate(cache, st)
        u, g = bvc.get_solution(st)
        outs.append((u.clone(), g.clone()))
    shape, ms = bvc.tune_gather(cache, st)
    torch.cuda.synchronize()
    print(f"[tune gather {dim}D] points per thread: boundary {shape[0]}, source {shape[1]}; {ms:.3f} ms")
    assert shape[0] in (2, 4, 6) and shape[1] in (2, 4) and ms > 0
    assert int(st.counts.sum().item()) == 0  # the tuner clears the state
    for u, g in outs[1:]:
        torch.testing.assert_close(u, outs[0][0], rtol=1e-10, atol=1e-12)
        torch.testing.assert_close(g, outs[0][1], rtol=1e-10, atol=1e-10)
    bvc.set_gather_shape(dim, 0, 0)
    bvc.set_gather_shape(dim, 1, 0)
    with pytest.raises(bvc.BvcError):
        bvc.set_gather_shape(dim, 1, 6)
