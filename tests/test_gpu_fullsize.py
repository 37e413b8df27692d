"""Full-size parity on the scale-22 R-MAT workload (4.19M vertices, 128M
directed edges; seed = vertex 0's highest-degree neighbour), in the launch
configuration bench.py times: Nibble (T=20, eps=1e-7), HK-PR (t=10, N=20,
eps=1e-7), rand-HK-PR (t=10, K=10, 1e6 walks, Philox 7) and PR-Nibble
(alpha=0.01, eps=1e-7), each followed by the sweep cut.  The oracle finishes
each of these in seconds on one core."""
import numpy as np
import pytest

import oracle
from paper_1604_07515_gb300 import inputs, lgc

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def big():
    off, col = inputs.rmat(22, seed=2)
    ctx = lgc.Context(0)
    ctx.set_option(lgc.OPT_TRACE, 1)
    g = lgc.Graph(ctx, off, col)
    x = inputs.config1_seed(off, col)
    yield ctx, g, off, col, x
    g.close()
    ctx.close()


def rel_l1(a_idx, a_val, b_idx, b_val, n):
    a, b = np.zeros(n), np.zeros(n)
    a[a_idx] = a_val
    b[b_idx] = b_val
    return np.abs(a - b).sum() / np.abs(b).sum()


def check_sweep(g, off, col, p, ref, exact=True):
    c = lgc.sweep(g, p)
    rs = oracle.sweep(off, col, ref.idx, ref.val)
    if exact:
        assert c.size == rs.best and c.vol == rs.best_vol and c.cut == rs.best_cut
        assert np.array_equal(c.ids, rs.cluster)
        assert c.conductance == rs.conductance
    else:
        assert abs(c.conductance - rs.conductance) <= 1e-9


def test_nibble_scale22(big):
    ctx, g, off, col, x = big
    ref = oracle.nibble(off, col, x, 20, 1e-7, trace=True)
    p, st = lgc.nibble(g, x, 20, 1e-7, mode="det")
    assert np.array_equal(p.idx, ref.idx) and np.array_equal(p.val, ref.val)
    assert [f.tolist() for f in ctx.trace()] == [f.tolist() for f in ref.trace]
    check_sweep(g, off, col, p, ref)
    p, st = lgc.nibble(g, x, 20, 1e-7, mode="atomic")
    assert rel_l1(p.idx, p.val, ref.idx, ref.val, len(off) - 1) <= 1e-12


def test_hkpr_scale22(big):
    ctx, g, off, col, x = big
    ref = oracle.hkpr(off, col, x, 10.0, 20, 1e-7)
    p, st = lgc.hkpr(g, x, 10.0, 20, 1e-7, mode="atomic")
    assert st.pushed_edges == ref.pushed_edges
    assert rel_l1(p.idx, p.val, ref.idx, ref.val, len(off) - 1) <= 1e-12
    check_sweep(g, off, col, p, ref, exact=False)
    p, st = lgc.hkpr(g, x, 10.0, 20, 1e-7, mode="det")
    assert np.array_equal(p.idx, ref.idx) and np.array_equal(p.val, ref.val)
    check_sweep(g, off, col, p, ref)


def test_rand_hkpr_scale22(big):
    ctx, g, off, col, x = big
    ref = oracle.rand_hkpr(off, col, x, 10.0, 10, 1_000_000, 7)
    p, st = lgc.rand_hkpr(g, x, 10.0, 10, 1_000_000, 7)
    assert np.array_equal(ctx.rand_hkpr_endpoints(1_000_000), ref.endpoints)
    assert np.array_equal(p.idx, ref.idx) and np.array_equal(p.val, ref.val)
    check_sweep(g, off, col, p, ref)


def test_prnibble_scale22(big):
    ctx, g, off, col, x = big
    ref = oracle.prnibble(off, col, x, 0.01, 1e-7, trace=True)
    p, st = lgc.prnibble(g, x, 0.01, 1e-7, mode="det")
    assert np.array_equal(p.idx, ref.idx) and np.array_equal(p.val, ref.val)
    assert [f.tolist() for f in ctx.trace()] == [f.tolist() for f in ref.trace]
    check_sweep(g, off, col, p, ref)
    p, st = lgc.prnibble(g, x, 0.01, 1e-7, mode="atomic")
    assert rel_l1(p.idx, p.val, ref.idx, ref.val, len(off) - 1) <= 1e-12
    check_sweep(g, off, col, p, ref, exact=False)
