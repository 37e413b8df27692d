"""PR-Nibble from a weighted seed set with beta-fraction rounds
(lgc_prnibble_set) against the oracle (orc_prnibble_set).  Deterministic
mode: p, r, rounds, pushes and every round's pushing set bit-identical;
atomic mode: p within 1e-12 relative L1."""
import numpy as np
import pytest

import oracle
from paper_1604_07515_gb300 import inputs, lgc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = lgc.Context(0)
    c.set_option(lgc.OPT_TRACE, 1)
    yield c
    c.close()


GRAPHS = {"rand500": lambda: inputs.random_graph(500, 2000, seed=3),
          "rmat13": lambda: inputs.rmat(13, seed=9),
          "rmat16": lambda: inputs.rmat(16, seed=1)}
_cache = {}


def graph(ctx, name):
    if name not in _cache:
        off, col = GRAPHS[name]()
        _cache[name] = (off, col, lgc.Graph(ctx, off, col))
    return _cache[name]


def seed_set(off, k, salt):
    cand = np.flatnonzero(np.diff(off) >= 1)
    rng = np.random.default_rng(salt)
    s = rng.choice(cand, size=k, replace=False).astype(np.int32)
    w = rng.uniform(0.2, 3.0, size=k)
    return s, w


def rel_l1(a_idx, a_val, b_idx, b_val):
    n = int(max(a_idx.max(initial=0), b_idx.max(initial=0))) + 1
    a, b = np.zeros(n), np.zeros(n)
    a[a_idx] = a_val
    b[b_idx] = b_val
    return np.abs(a - b).sum() / np.abs(b).sum()


@pytest.mark.parametrize("rule", ["opt", "orig"])
@pytest.mark.parametrize("beta", [1.0, 0.5, 0.1, 1e-9])
@pytest.mark.parametrize("k", [1, 3, 8])
@pytest.mark.parametrize("name,alpha,eps", [("rand500", 0.05, 1e-5), ("rmat13", 0.05, 1e-6),
                                            ("rmat16", 0.01, 1e-5)])
def test_prnibble_set_det_bitexact(ctx, name, alpha, eps, k, beta, rule):
    off, col, g = graph(ctx, name)
    s, w = seed_set(off, k, 100 + k)
    if beta == 1e-9:
        eps = max(eps * 100, 1e-4)  # one vertex per round: keep the round count small
    ref = oracle.prnibble_set(off, col, s, w, alpha, eps, rule=0 if rule == "opt" else 1,
                              beta=beta, trace=True)
    p, st = lgc.prnibble_set(g, s, alpha, eps, weights=w, beta=beta, rule=rule, mode="det")
    assert (st.rounds, st.pushes, st.pushed_edges) == (ref.rounds, ref.pushes, ref.pushed_edges)
    assert np.array_equal(p.idx, ref.idx) and np.array_equal(p.val, ref.val)
    r = ctx.residual()
    assert np.array_equal(r.idx, ref.idx2) and np.array_equal(r.val, ref.val2)
    tr = ctx.trace()
    assert len(tr) == len(ref.trace)
    for a, b in zip(tr, ref.trace):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("beta", [1.0, 0.5])
@pytest.mark.parametrize("name", ["rand500", "rmat13", "rmat16"])
def test_prnibble_set_atomic(ctx, name, beta):
    off, col, g = graph(ctx, name)
    for k in (1, 4):
        s, w = seed_set(off, k, 7 + k)
        ref = oracle.prnibble_set(off, col, s, w, 0.02, 1e-6, beta=beta)
        p, st = lgc.prnibble_set(g, s, 0.02, 1e-6, weights=w, beta=beta, mode="atomic")
        assert st.pushed_edges == ref.pushed_edges
        assert rel_l1(p.idx, p.val, ref.idx, ref.val) <= 1e-12


def test_prnibble_set_one_seed_equals_prnibble(ctx):
    off, col, g = graph(ctx, "rmat13")
    x = inputs.config1_seed(off, col)
    a, sa = lgc.prnibble(g, x, 0.01, 1e-6, mode="det")
    b, sb = lgc.prnibble_set(g, [x], 0.01, 1e-6, mode="det")
    assert np.array_equal(a.idx, b.idx) and np.array_equal(a.val, b.val)
    assert (sa.rounds, sa.pushes) == (sb.rounds, sb.pushes)


def test_prnibble_set_errors(ctx):
    off, col, g = graph(ctx, "rmat13")
    x = inputs.config1_seed(off, col)
    iso = int(np.flatnonzero(np.diff(off) == 0)[0])
    for seeds, w, beta in [([x, x], None, 1.0), ([x], [0.0], 1.0), ([x], None, 0.0),
                           ([x], None, 1.5), ([x, iso], None, 1.0), ([len(off)], None, 1.0)]:
        with pytest.raises(lgc.LgcError):
            lgc.prnibble_set(g, seeds, 0.01, 1e-5, weights=w, beta=beta)
    with pytest.raises(lgc.LgcError):
        lgc.prnibble_set(g, [], 0.01, 1e-5)
