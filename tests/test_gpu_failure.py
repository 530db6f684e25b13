"""Failure detection on the GPU without a fault: the gathers' bounded wait
for a tile copy, cut short in a self-test kernel whose barrier nothing
completes, gives up, records the status bit the host reads, and the kernel
returns -- the context stays usable for the next solve."""
import time

import numpy as np
import pytest
import torch

from paper_2302_11825_gb300 import bvc
from paper_2302_11825_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def _small_solve():
    w = wl.circle_laplace(n_samples=256, walks=16)
    geom = bvc.Geometry(w.V, w.F)
    opts = bvc.cache_opts(w.n_samples, w.walks, w.offset_l, w.eps, seed=0)
    cache = bvc.cache_build(geom, w.g, w.f, opts, bvc.Cache(2, w.n_samples))
    st = bvc.EvalState(bvc.soa(w.eval_pts[:300]))
    bvc.evaluate(cache, st)
    u, _ = bvc.get_solution(st)
    torch.cuda.synchronize()
    return u.cpu().numpy()


def test_bounded_wait_gives_up_and_the_context_stays_usable():
    before = _small_solve()
    bvc.gather_status(reset=True)
    t0 = time.perf_counter()
    bvc.wait_selftest(2_000_000)  # 2 ms
    flags, st = bvc.gather_status()
    elapsed = time.perf_counter() - t0
    assert flags & 2, flags           # the wait ran out and said so
    assert not flags & 1              # no real tile copy stalled
    assert st == bvc.OK
    assert elapsed < 5.0
    bvc.gather_status(reset=True)
    # the context is intact: the same solve gives the same bits
    after = _small_solve()
    assert np.all(np.isfinite(after))
    np.testing.assert_array_equal(before, after)
    flags, st = bvc.gather_status(reset=True)
    assert flags == 0 and st == bvc.OK
