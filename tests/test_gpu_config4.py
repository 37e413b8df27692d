"""Parity of the batched engine on the many-seed workload: R-MAT scale 24
(16.8M vertices, edge factor 16, seed 4), PR-Nibble alpha = 0.01 from seeds
drawn uniformly among vertices of degree >= 2 (stream 4) with eps
log-uniform in [1e-8, 1e-5] (stream 4) -- the seeds bench.py times.  A
subset of them (every 16th, 64 seeds, deterministic mode; and 32 others in
atomic mode) runs in one lgc_prnibble_batch call each and is compared with
the oracle seed by seed, with its sweep cut from lgc_sweep_batch."""
import numpy as np
import pytest

import oracle
from paper_1604_07515_gb300 import inputs, lgc

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def many():
    off, col = inputs.rmat(24, seed=4)
    ctx = lgc.Context(0)
    g = lgc.Graph(ctx, off, col)
    seeds = inputs.seeds_deg2(off, 1024, 4)
    eps = inputs.eps_loguniform(1024, 4, -8.0, -5.0)
    yield ctx, g, off, col, seeds, eps
    g.close()
    ctx.close()


def rel_l1(a_idx, a_val, b_idx, b_val):
    n = int(max(a_idx.max(initial=0), b_idx.max(initial=0))) + 1
    a, b = np.zeros(n), np.zeros(n)
    a[a_idx] = a_val
    b[b_idx] = b_val
    return np.abs(a - b).sum() / np.abs(b).sum()


def test_config4_batched_det(many):
    ctx, g, off, col, seeds, eps = many
    sel = np.arange(0, 1024, 16)
    ps, sts = lgc.prnibble_batch(g, seeds[sel], 0.01, eps[sel], mode="det")
    cs = lgc.sweep_batch(g, ps)
    for k, b in enumerate(sel):
        ref = oracle.prnibble(off, col, int(seeds[b]), 0.01, float(eps[b]))
        assert (sts[k].rounds, sts[k].pushes, sts[k].pushed_edges) == (ref.rounds, ref.pushes,
                                                                       ref.pushed_edges)
        assert np.array_equal(ps[k].idx, ref.idx) and np.array_equal(ps[k].val, ref.val)
        rs = oracle.sweep(off, col, ref.idx, ref.val)
        assert cs[k].size == rs.best and cs[k].vol == rs.best_vol and cs[k].cut == rs.best_cut
        assert np.array_equal(cs[k].ids, rs.cluster)


def test_config4_batched_atomic(many):
    ctx, g, off, col, seeds, eps = many
    sel = np.arange(8, 1024, 32)
    ps, sts = lgc.prnibble_batch(g, seeds[sel], 0.01, eps[sel], mode="atomic")
    cs = lgc.sweep_batch(g, ps)
    for k, b in enumerate(sel):
        ref = oracle.prnibble(off, col, int(seeds[b]), 0.01, float(eps[b]))
        assert sts[k].pushed_edges == ref.pushed_edges
        assert rel_l1(ps[k].idx, ps[k].val, ref.idx, ref.val) <= 1e-12
        rs = oracle.sweep(off, col, ref.idx, ref.val)
        assert abs(cs[k].conductance - rs.conductance) <= 1e-9
