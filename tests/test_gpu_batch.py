"""lgc_prnibble_batch: many seeds advance together, one launch per kernel per
round.  Each seed's result must equal its single-seed result (bit-identical
in deterministic mode, within 1e-12 relative L1 in atomic mode) and the
oracle's."""
import numpy as np
import pytest

import oracle
from paper_1604_07515_gb300 import inputs, lgc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    ctx = lgc.Context(0)
    graphs = {}
    for name, (s, seed) in {"rmat13": (13, 9), "rmat16": (16, 1)}.items():
        off, col = inputs.rmat(s, seed=seed)
        graphs[name] = (off, col, lgc.Graph(ctx, off, col))
    yield ctx, graphs
    ctx.close()


def rel_l1(a_idx, a_val, b_idx, b_val):
    n = int(max(a_idx.max(initial=0), b_idx.max(initial=0))) + 1
    a, b = np.zeros(n), np.zeros(n)
    a[a_idx] = a_val
    b[b_idx] = b_val
    return np.abs(a - b).sum() / np.abs(b).sum()


@pytest.mark.parametrize("name", ["rmat13", "rmat16"])
@pytest.mark.parametrize("mode", ["det", "atomic"])
def test_batch_equals_single_seed(setup, name, mode):
    ctx, graphs = setup
    off, col, g = graphs[name]
    B = 40
    seeds = inputs.seeds_deg2(off, B, 11)
    eps = inputs.eps_loguniform(B, 12, -6.5, -4.0)
    alpha = np.where(np.arange(B) % 3 == 0, 0.05, 0.01)
    ps, sts = lgc.prnibble_batch(g, seeds, alpha, eps, mode=mode)
    for b in range(B):
        p1, st1 = lgc.prnibble(g, int(seeds[b]), float(alpha[b]), float(eps[b]), mode=mode)
        ref = oracle.prnibble(off, col, int(seeds[b]), float(alpha[b]), float(eps[b]))
        assert sts[b].rounds == ref.rounds and sts[b].pushed_edges == ref.pushed_edges
        if mode == "det":
            assert np.array_equal(ps[b].idx, p1.idx) and np.array_equal(ps[b].val, p1.val)
            assert np.array_equal(ps[b].idx, ref.idx) and np.array_equal(ps[b].val, ref.val)
        else:
            assert rel_l1(ps[b].idx, ps[b].val, ref.idx, ref.val) <= 1e-12


def test_batch_original_rule_and_round_limit(setup):
    ctx, graphs = setup
    off, col, g = graphs["rmat13"]
    seeds = inputs.seeds_deg2(off, 9, 21)
    ps, sts = lgc.prnibble_batch(g, seeds, 0.05, 1e-5, rule="orig", mode="det", max_rounds=3)
    for b in range(9):
        ref = oracle.prnibble(off, col, int(seeds[b]), 0.05, 1e-5, rule=1, max_rounds=3)
        assert np.array_equal(ps[b].idx, ref.idx) and np.array_equal(ps[b].val, ref.val)
        assert sts[b].rounds == ref.rounds


def test_batch_duplicate_seeds_and_errors(setup):
    ctx, graphs = setup
    off, col, g = graphs["rmat13"]
    x = inputs.config1_seed(off, col)
    ps, sts = lgc.prnibble_batch(g, [x, x, x], 0.01, 1e-5, mode="det")
    assert all(np.array_equal(ps[0].val, p.val) for p in ps)
    iso = int(np.flatnonzero(np.diff(off) == 0)[0])
    with pytest.raises(lgc.LgcError):
        lgc.prnibble_batch(g, [x, iso], 0.01, 1e-5)
    with pytest.raises(lgc.LgcError):
        lgc.prnibble_batch(g, [x, x], [0.01, 1.5], 1e-5)
