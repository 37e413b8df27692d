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


@pytest.mark.parametrize("handoff", [200, 3000])
@pytest.mark.parametrize("rule", ["opt", "orig"])
@pytest.mark.parametrize("mode", ["det", "atomic"])
def test_batch_handoff_to_single_seed(setup, handoff, rule, mode):
    """Seeds whose frontier passes LGC_OPT_BATCH_HANDOFF edges finish alone
    from the state the batch left: results and counters as in one
    uninterrupted run (det bit-identical to the oracle), round limits
    included."""
    ctx, graphs = setup
    off, col, g = graphs["rmat16"]
    B = 24
    seeds = inputs.seeds_deg2(off, B, 31)
    eps = inputs.eps_loguniform(B, 32, -7.0, -4.5)
    ctx.set_option(lgc.OPT_BATCH_HANDOFF, handoff)
    try:
        prm_alpha = 0.01
        ps, sts = lgc.prnibble_batch(g, seeds, prm_alpha, eps, rule=rule, mode=mode)
        for b in range(B):
            ref = oracle.prnibble(off, col, int(seeds[b]), prm_alpha, float(eps[b]),
                                  rule=0 if rule == "opt" else 1)
            assert (sts[b].rounds, sts[b].pushes, sts[b].pushed_edges) == (
                ref.rounds, ref.pushes, ref.pushed_edges)
            if mode == "det":
                assert np.array_equal(ps[b].idx, ref.idx) and np.array_equal(ps[b].val, ref.val)
            else:
                assert rel_l1(ps[b].idx, ps[b].val, ref.idx, ref.val) <= 1e-12
        # round limits across the hand-off
        for b, k in ((3, 2), (5, 6)):
            p1, s1 = lgc.prnibble_batch(g, seeds[b:b + 2], prm_alpha, eps[b:b + 2], rule=rule,
                                        mode=mode, max_rounds=k)
            for j in range(2):
                ref = oracle.prnibble(off, col, int(seeds[b + j]), prm_alpha, float(eps[b + j]),
                                      rule=0 if rule == "opt" else 1, max_rounds=k)
                assert s1[j].rounds == ref.rounds and s1[j].pushed_edges == ref.pushed_edges
                if mode == "det":
                    assert np.array_equal(p1[j].idx, ref.idx)
                    assert np.array_equal(p1[j].val, ref.val)
                else:
                    assert rel_l1(p1[j].idx, p1[j].val, ref.idx, ref.val) <= 1e-12
    finally:
        ctx.set_option(lgc.OPT_BATCH_HANDOFF, 0)


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


def same_cluster(c, ref):
    assert c.size == ref.best and c.vol == ref.best_vol and c.cut == ref.best_cut
    assert np.array_equal(c.ids, ref.cluster)
    assert c.conductance == ref.conductance or (np.isinf(c.conductance)
                                                and np.isinf(ref.conductance))


@pytest.mark.parametrize("on_device", [False, True])
def test_sweep_batch_equals_oracle(setup, on_device):
    """lgc_sweep_batch over PR-Nibble vectors and hand-made ones (empty, all
    zero, ties in p/d, the whole support) gives each vector's own sweep."""
    ctx, graphs = setup
    off, col, g = graphs["rmat16"]
    d = np.diff(off)
    seeds = inputs.seeds_deg2(off, 24, 31)
    eps = inputs.eps_loguniform(24, 32, -6.0, -4.0)
    ctx.set_option(lgc.OPT_RESULT_ON_DEVICE, 1 if on_device else 0)
    try:
        ps, _ = lgc.prnibble_batch(g, seeds, 0.05, eps, mode="det")
        vecs = list(ps)
        host = []
        for p in ps:
            r = oracle.prnibble(off, col, int(seeds[len(host)]), 0.05, float(eps[len(host)]))
            host.append((r.idx, r.val))
        rng = np.random.default_rng(3)
        sup = np.flatnonzero(d > 0).astype(np.int32)
        extra = [(np.zeros(0, np.int32), np.zeros(0)), (sup[:5], np.zeros(5)),
                 (sup[:300], (rng.integers(0, 4, 300) * 0.25 * d[sup[:300]])),
                 (sup, np.ones(len(sup)))]
        for idx, val in extra:
            vecs.insert(int(rng.integers(0, len(vecs) + 1)), lgc.host_svec(idx, val))
        cs = lgc.sweep_batch(g, vecs)
        assert len(cs) == len(vecs)
        for v, c in zip(vecs, cs):
            c1 = lgc.sweep(g, v)
            assert (c.size, c.vol, c.cut) == (c1.size, c1.vol, c1.cut)
            assert c.conductance == c1.conductance or (np.isinf(c.conductance)
                                                       and np.isinf(c1.conductance))
            if not on_device:
                assert np.array_equal(c.ids, c1.ids)
        if not on_device:
            for k, (idx, val) in enumerate(host):
                same_cluster(cs[vecs.index(ps[k])], oracle.sweep(off, col, idx, val))
            for idx, val in extra:
                c = [c for v, c in zip(vecs, cs) if v.nnz == len(idx) and not v.on_device
                     and np.array_equal(v.idx, idx) and np.array_equal(v.val, val)][0]
                same_cluster(c, oracle.sweep(off, col, idx, val))
    finally:
        ctx.set_option(lgc.OPT_RESULT_ON_DEVICE, 0)


def test_sweep_batch_rejects_bad_entries(setup):
    ctx, graphs = setup
    off, col, g = graphs["rmat13"]
    iso = int(np.flatnonzero(np.diff(off) == 0)[0])
    good = lgc.host_svec([int(np.flatnonzero(np.diff(off) > 0)[0])], [1.0])
    with pytest.raises(lgc.LgcError):
        lgc.sweep_batch(g, [good, lgc.host_svec([iso], [0.5])])
    with pytest.raises(lgc.LgcError):
        lgc.sweep_batch(g, [good, lgc.host_svec([len(off) + 5], [0.5])])
    assert lgc.sweep_batch(g, []) == []
