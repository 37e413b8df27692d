"""Parity on the largest PR-Nibble workload: R-MAT scale 26 (67.1M vertices,
edge factor 16, a=0.57 b=c=0.19, seed 3; about 2.1 billion directed CSR
entries, int32 ids, int64 offsets), PR-Nibble alpha=0.01 at eps 1e-7 and
1e-8 from seeds drawn uniformly among vertices of degree >= 2, one seed per
call, each followed by the sweep cut.  Deterministic mode: p, rounds and
pushes bit-identical to the oracle and the same cluster; atomic mode: p
within 1e-12 relative L1 and the conductance within 1e-9.  The seeds'
diffusions stay local, so the oracle finishes each in seconds."""
import numpy as np
import pytest

import oracle
from paper_1604_07515_gb300 import inputs, lgc

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def huge():
    off, col = inputs.rmat(26, seed=3)
    ctx = lgc.Context(0)
    g = lgc.Graph(ctx, off, col)
    seeds = inputs.seeds_deg2(off, 4, 3)
    yield ctx, g, off, col, seeds
    g.close()
    ctx.close()


def test_graph_shape(huge):
    ctx, g, off, col, seeds = huge
    assert len(off) - 1 == 1 << 26
    assert g.nnz == len(col) and g.nnz > 2_000_000_000
    assert off.dtype == np.int64 and col.dtype == np.int32


def rel_l1(a_idx, a_val, b_idx, b_val):
    n = int(max(a_idx.max(initial=0), b_idx.max(initial=0))) + 1
    a, b = np.zeros(n), np.zeros(n)
    a[a_idx] = a_val
    b[b_idx] = b_val
    return np.abs(a - b).sum() / np.abs(b).sum()


@pytest.mark.parametrize("eps", [1e-7, 1e-8])
def test_config3_det(huge, eps):
    ctx, g, off, col, seeds = huge
    for x in seeds[:2]:
        ref = oracle.prnibble(off, col, int(x), 0.01, eps)
        p, st = lgc.prnibble(g, int(x), 0.01, eps, mode="det")
        assert (st.rounds, st.pushes, st.pushed_edges) == (ref.rounds, ref.pushes,
                                                           ref.pushed_edges)
        assert np.array_equal(p.idx, ref.idx) and np.array_equal(p.val, ref.val)
        c = lgc.sweep(g, p)
        rs = oracle.sweep(off, col, ref.idx, ref.val)
        assert c.size == rs.best and c.vol == rs.best_vol and c.cut == rs.best_cut
        assert np.array_equal(c.ids, rs.cluster) and c.conductance == rs.conductance


@pytest.mark.parametrize("eps", [1e-7, 1e-8])
def test_config3_atomic(huge, eps):
    ctx, g, off, col, seeds = huge
    for x in seeds[2:]:
        ref = oracle.prnibble(off, col, int(x), 0.01, eps)
        p, st = lgc.prnibble(g, int(x), 0.01, eps, mode="atomic")
        assert st.rounds == ref.rounds and st.pushed_edges == ref.pushed_edges
        assert rel_l1(p.idx, p.val, ref.idx, ref.val) <= 1e-12
        c = lgc.sweep(g, p)
        rs = oracle.sweep(off, col, ref.idx, ref.val)
        assert abs(c.conductance - rs.conductance) <= 1e-9
