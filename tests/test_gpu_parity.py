"""GPU parity: the CUDA library (through the C ABI) against the CPU oracle.

Deterministic mode: p, r, every frontier, rounds and push counts must be
bit-identical.  Atomic mode: p within 1e-12 relative L1 of the oracle and the
sweep's conductance within 1e-9.  The sweep cut and rand-HK-PR endpoints are
exact.  Sizes span many CTA tiles with ragged tails; the scale-16 and
scale-22 R-MAT graphs are the two smallest benchmark workloads in full."""
import math

import numpy as np
import pytest

import oracle
from paper_1604_07515_gb300 import inputs, lgc

pytestmark = pytest.mark.gpu

ATOL_REL_L1 = 1e-12
PHI_TOL = 1e-9


@pytest.fixture(scope="module")
def ctx():
    c = lgc.Context(0)
    c.set_trace(1)  # lgc_set_trace(ctx, LGC_TRACE_FRONTIERS)
    yield c
    c.close()


@pytest.fixture(params=[0, 1, 2], ids=["auto", "hashed", "dense"])
def form(request, ctx):
    """Sparse-set representation: automatic, always hashed, always dense."""
    ctx.set_option(lgc.OPT_TABLE_FORM, request.param)
    yield request.param
    ctx.set_option(lgc.OPT_TABLE_FORM, 0)


_graph_cache = {}


def gpu_graph(ctx, name):
    if name not in _graph_cache:
        off, col = GRAPHS[name]()
        _graph_cache[name] = (off, col, lgc.Graph(ctx, off, col, validate=True))
    return _graph_cache[name]


GRAPHS = {
    "paper": inputs.paper_example,
    "path9": lambda: inputs.path(9),
    "star40": lambda: inputs.star(40),
    "cliques6": lambda: inputs.clique_pair(6),
    "grid6": lambda: inputs.grid3d(6),
    "rand500": lambda: inputs.random_graph(500, 2000, seed=3),
    "rmat10": lambda: inputs.rmat(10, seed=5),
    "rmat13": lambda: inputs.rmat(13, seed=9),
    "rmat16": lambda: inputs.rmat(16, seed=1),
}


def seeds_for(off, col, k=3, salt=0):
    s = [inputs.config1_seed(off, col)]
    s += inputs.seeds_deg2(off, k - 1, 1000 + salt).tolist() if (np.diff(off) >= 2).any() else []
    return s


def rel_l1(idx_a, val_a, idx_b, val_b):
    n = int(max(idx_a.max(initial=0), idx_b.max(initial=0))) + 1
    a = np.zeros(n)
    b = np.zeros(n)
    a[idx_a] = val_a
    b[idx_b] = val_b
    return np.abs(a - b).sum() / max(np.abs(b).sum(), 1e-300)


def assert_trace_equal(got, ref_trace):
    assert len(got) == len(ref_trace)
    for k, (f, r) in enumerate(zip(got, ref_trace)):
        assert np.array_equal(f, r), f"frontier of round {k} differs"


# ---------------------------------------------------------------------------
# sweep cut
# ---------------------------------------------------------------------------
def test_sweep_paper_example(ctx):
    off, col, g = gpu_graph(ctx, "paper")
    c = lgc.sweep(g, lgc.host_svec([0, 1, 2, 3], [0.4, 0.3, 0.3, 0.2]))
    assert c.ids.tolist() == [0, 1, 2] and c.vol == 7 and c.cut == 1
    assert c.conductance == 1.0 / 7.0


@pytest.mark.parametrize("name", ["rand500", "rmat10", "rmat13", "rmat16"])
def test_sweep_matches_oracle(ctx, name):
    off, col, g = gpu_graph(ctx, name)
    n = len(off) - 1
    d = np.diff(off)
    rng = np.random.default_rng(7)
    for trial in range(6):
        k = int(rng.integers(1, n))
        idx = np.sort(rng.choice(np.flatnonzero(d > 0), size=min(k, int((d > 0).sum())),
                                 replace=False)).astype(np.int32)
        if trial % 2 == 0:  # coarse values: many ties in p/d
            val = rng.integers(0, 5, size=len(idx)) * 0.125 * d[idx]
        else:
            val = rng.random(len(idx)) ** 3
        ref = oracle.sweep(off, col, idx, val)
        # both forms of the crossing counts (edge-balanced, vertex-centric)
        try:
            for form in (0, 1, 2):
                ctx.set_option(lgc.OPT_SWEEP_CROSS, form)
                c = lgc.sweep(g, lgc.host_svec(idx, val))
                assert c.size == ref.best
                assert c.vol == ref.best_vol and c.cut == ref.best_cut
                assert np.array_equal(c.ids, ref.cluster)
                assert c.conductance == ref.conductance or (math.isinf(c.conductance)
                                                            and math.isinf(ref.conductance))
        finally:
            ctx.set_option(lgc.OPT_SWEEP_CROSS, 0)


@pytest.mark.parametrize("pattern", ["low_byte", "low_two_bytes", "all_equal"])
def test_sweep_sort_digit_patterns(ctx, pattern):
    """Sort keys whose 8-bit digits are uniform in all but the lowest one
    (one digit pass runs: the result ends in the scratch buffers and is
    copied back), all but the lowest two, or in every digit (no pass runs;
    equal keys keep ascending id), over several sort tiles (p/d on the
    degree-1 vertices of R-MAT 16, so p/d is p exactly), in both forms of
    the crossing counts: the oracle's cut, bit for bit."""
    off, col, g = gpu_graph(ctx, "rmat16")
    d = np.diff(off)
    idx = np.flatnonzero(d == 1).astype(np.int32)
    assert len(idx) > 4 * 2048
    rng = np.random.default_rng(11)
    if pattern == "all_equal":
        val = np.full(len(idx), 0.25)
    else:
        span = 256 if pattern == "low_byte" else 65536
        val = 0.5 + rng.integers(0, span, size=len(idx)).astype(np.float64) * 2.0 ** -53
    ref = oracle.sweep(off, col, idx, val)
    try:
        for form in (0, 1):
            ctx.set_option(lgc.OPT_SWEEP_CROSS, form)
            c = lgc.sweep(g, lgc.host_svec(idx, val))
            assert (c.size, c.vol, c.cut) == (ref.best, ref.best_vol, ref.best_cut)
            assert np.array_equal(c.ids, ref.cluster)
            assert c.conductance == ref.conductance
    finally:
        ctx.set_option(lgc.OPT_SWEEP_CROSS, 0)


@pytest.mark.parametrize("n0", [1024, 1025, 2047, 2048, 2049, 4097, 6145])
def test_sweep_at_tile_boundaries(ctx, n0):
    """Supports of sizes around the small-sort limit (1024), the sort and
    scan tiles (2048) and a few tiles more: the sort, the volume and cut
    scans and the crossing counts in both forms give the oracle's cut."""
    off, col, g = gpu_graph(ctx, "rmat16")
    d = np.diff(off)
    rng = np.random.default_rng(n0)
    idx = np.sort(rng.choice(np.flatnonzero(d > 0), size=n0, replace=False)).astype(np.int32)
    val = rng.random(n0) ** 2
    ref = oracle.sweep(off, col, idx, val)
    try:
        for form in (1, 2):
            ctx.set_option(lgc.OPT_SWEEP_CROSS, form)
            c = lgc.sweep(g, lgc.host_svec(idx, val))
            assert (c.size, c.vol, c.cut) == (ref.best, ref.best_vol, ref.best_cut)
            assert np.array_equal(c.ids, ref.cluster)
            assert c.conductance == ref.conductance
    finally:
        ctx.set_option(lgc.OPT_SWEEP_CROSS, 0)


def test_sweep_edge_cases(ctx):
    off, col, g = gpu_graph(ctx, "cliques6")
    n = len(off) - 1
    c = lgc.sweep(g, lgc.host_svec(np.zeros(0, np.int32), np.zeros(0)))
    assert c.size == 0 and math.isinf(c.conductance)
    c = lgc.sweep(g, lgc.host_svec([3], [0.0]))  # zeros are not in the support
    assert c.size == 0
    ref = oracle.sweep(off, col, np.arange(n), np.ones(n))
    c = lgc.sweep(g, lgc.host_svec(np.arange(n), np.ones(n)))
    assert c.size == ref.best and c.cut == ref.best_cut and c.vol == ref.best_vol


def test_sweep_rejects_invalid_entries(ctx):
    """A vertex named twice is LGC_EINVAL, single and batched, with the rank
    hash table (small input) and the dense rank array (input over n/64,
    whose volume then exceeds 2m); the context stays usable."""
    off, col, g = gpu_graph(ctx, "rmat13")
    d = np.diff(off)
    v = np.flatnonzero(d > 0).astype(np.int32)
    small = lgc.host_svec(np.array([v[0], v[1], v[0]], np.int32), [0.3, 0.2, 0.1])
    big_idx = np.concatenate([v, v[:5]]).astype(np.int32)
    big = lgc.host_svec(big_idx, np.ones(len(big_idx)))
    ok = lgc.host_svec(v[2:3], [1.0])
    for p in (small, big):
        with pytest.raises(lgc.LgcError) as e:
            lgc.sweep(g, p)
        assert e.value.status == lgc.LGC_EINVAL
        with pytest.raises(lgc.LgcError) as e:
            lgc.sweep_batch(g, [ok, p])
        assert e.value.status == lgc.LGC_EINVAL
    with pytest.raises(lgc.LgcError) as e:
        lgc.sweep(g, lgc.host_svec(np.array([len(off) - 1], np.int32), [1.0]))  # not a vertex
    assert e.value.status == lgc.LGC_EINVAL
    ref = oracle.sweep(off, col, v, np.ones(len(v)))
    c = lgc.sweep(g, lgc.host_svec(v, np.ones(len(v))))
    assert c.size == ref.best and c.cut == ref.best_cut and c.vol == ref.best_vol


# ---------------------------------------------------------------------------
# PR-Nibble
# ---------------------------------------------------------------------------
PR_CASES = [("paper", 0.15, 1e-4), ("path9", 0.1, 1e-5), ("star40", 0.05, 1e-4),
            ("cliques6", 0.1, 1e-6), ("grid6", 0.05, 1e-6), ("rand500", 0.02, 1e-6),
            ("rmat10", 0.01, 1e-5), ("rmat13", 0.01, 1e-6)]


@pytest.mark.parametrize("rule", ["opt", "orig"])
@pytest.mark.parametrize("name,alpha,eps", PR_CASES)
def test_prnibble_det_bitexact(ctx, form, name, alpha, eps, rule):
    off, col, g = gpu_graph(ctx, name)
    for x in seeds_for(off, col, 2):
        ref = oracle.prnibble(off, col, x, alpha, eps, rule=1 if rule == "orig" else 0,
                              trace=True)
        p, st = lgc.prnibble(g, x, alpha, eps, rule=rule, mode="det")
        assert np.array_equal(p.idx, ref.idx)
        assert np.array_equal(p.val, ref.val), "p differs"
        r = ctx.residual()
        assert np.array_equal(r.idx, ref.idx2)
        assert np.array_equal(r.val, ref.val2), "r differs"
        assert_trace_equal(ctx.trace(), ref.trace)
        assert (st.rounds, st.pushes, st.pushed_edges, st.touched) == (
            ref.rounds, ref.pushes, ref.pushed_edges, ref.touched)


@pytest.mark.parametrize("name,alpha,eps", PR_CASES)
def test_prnibble_atomic_within_tolerance(ctx, form, name, alpha, eps):
    off, col, g = gpu_graph(ctx, name)
    for x in seeds_for(off, col, 2):
        ref = oracle.prnibble(off, col, x, alpha, eps)
        p, st = lgc.prnibble(g, x, alpha, eps, mode="atomic")
        assert rel_l1(p.idx, p.val, ref.idx, ref.val) <= ATOL_REL_L1
        c = lgc.sweep(g, p)
        rs = oracle.sweep(off, col, ref.idx, ref.val)
        assert abs(c.conductance - rs.conductance) <= PHI_TOL
        # the atomic frontiers are the same sets, in arrival order
        tr = ctx.trace()
        rt = oracle.prnibble(off, col, x, alpha, eps, trace=True).trace
        assert [np.sort(f).tolist() for f in tr] == [f.tolist() for f in rt]


def test_prnibble_config1_full_size(ctx):
    """Scale-16 R-MAT, seed = vertex 0's highest-degree neighbour, alpha 0.01,
    eps 1e-6, deterministic mode: bit-exact p, r, frontiers; exact sweep."""
    off, col, g = gpu_graph(ctx, "rmat16")
    x = inputs.config1_seed(off, col)
    ref = oracle.prnibble(off, col, x, 0.01, 1e-6, trace=True)
    p, st = lgc.prnibble(g, x, 0.01, 1e-6, mode="det")
    assert np.array_equal(p.idx, ref.idx) and np.array_equal(p.val, ref.val)
    r = ctx.residual()
    assert np.array_equal(r.idx, ref.idx2) and np.array_equal(r.val, ref.val2)
    assert_trace_equal(ctx.trace(), ref.trace)
    c = lgc.sweep(g, p)
    rs = oracle.sweep(off, col, ref.idx, ref.val)
    assert np.array_equal(c.ids, rs.cluster) and c.vol == rs.best_vol and c.cut == rs.best_cut
    assert c.conductance == rs.conductance


def test_prnibble_invalid_inputs(ctx):
    off, col, g = gpu_graph(ctx, "rmat10")
    iso = int(np.flatnonzero(np.diff(off) == 0)[0])
    for seed in (-1, len(off) - 1, iso):
        with pytest.raises(lgc.LgcError) as e:
            lgc.prnibble(g, seed, 0.01, 1e-5)
        assert e.value.status == lgc.LGC_EINVAL
    for alpha, eps in [(0.0, 1e-5), (1.0, 1e-5), (0.1, 0.0), (0.1, -1.0)]:
        with pytest.raises(lgc.LgcError):
            lgc.prnibble(g, 1, alpha, eps)


def test_prnibble_max_rounds(ctx):
    off, col, g = gpu_graph(ctx, "rmat13")
    x = inputs.config1_seed(off, col)
    for k in (1, 2, 3):
        ref = oracle.prnibble(off, col, x, 0.01, 1e-6, max_rounds=k)
        p, st = lgc.prnibble(g, x, 0.01, 1e-6, mode="det", max_rounds=k)
        assert st.rounds == k
        assert np.array_equal(p.idx, ref.idx) and np.array_equal(p.val, ref.val)


# ---------------------------------------------------------------------------
# Nibble
# ---------------------------------------------------------------------------
NIB_CASES = [("paper", 5, 1e-3), ("path9", 12, 1e-3), ("grid6", 8, 1e-4),
             ("rand500", 10, 1e-5), ("rmat10", 20, 1e-5), ("rmat13", 20, 1e-6),
             ("rmat13", 4, 0.0)]


@pytest.mark.parametrize("name,T,eps", NIB_CASES)
def test_nibble_det_bitexact(ctx, form, name, T, eps):
    off, col, g = gpu_graph(ctx, name)
    for x in seeds_for(off, col, 2, salt=1):
        ref = oracle.nibble(off, col, x, T, eps, trace=True)
        p, st = lgc.nibble(g, x, T, eps, mode="det")
        assert np.array_equal(p.idx, ref.idx)
        assert np.array_equal(p.val, ref.val)
        assert_trace_equal(ctx.trace(), ref.trace)
        assert (st.rounds, st.pushes, st.pushed_edges) == (ref.rounds, ref.pushes,
                                                            ref.pushed_edges)


@pytest.mark.parametrize("name,T,eps", NIB_CASES)
def test_nibble_atomic_within_tolerance(ctx, form, name, T, eps):
    off, col, g = gpu_graph(ctx, name)
    for x in seeds_for(off, col, 2, salt=1):
        ref = oracle.nibble(off, col, x, T, eps)
        p, st = lgc.nibble(g, x, T, eps, mode="atomic")
        assert rel_l1(p.idx, p.val, ref.idx, ref.val) <= ATOL_REL_L1


def test_nibble_early_exit(ctx):
    off, col, g = gpu_graph(ctx, "path9")
    ref = oracle.nibble(off, col, 0, 10, 0.3)
    for mode in ("det", "atomic"):
        p, st = lgc.nibble(g, 0, 10, 0.3, mode=mode)
        assert p.idx.tolist() == ref.idx.tolist() and p.val.tolist() == ref.val.tolist()


# ---------------------------------------------------------------------------
# HK-PR
# ---------------------------------------------------------------------------
HK_CASES = [("paper", 2.0, 6, 1e-3), ("grid6", 3.0, 10, 1e-4), ("rand500", 5.0, 12, 1e-4),
            ("rmat10", 5.0, 15, 1e-5), ("rmat13", 10.0, 20, 1e-7), ("rmat13", 3.0, 5, 0.0),
            ("cliques6", 1.0, 1, 1e-3)]


@pytest.mark.parametrize("name,t,N,eps", HK_CASES)
def test_hkpr_det_bitexact(ctx, form, name, t, N, eps):
    off, col, g = gpu_graph(ctx, name)
    for x in seeds_for(off, col, 2, salt=2):
        ref = oracle.hkpr(off, col, x, t, N, eps, trace=True)
        p, st = lgc.hkpr(g, x, t, N, eps, mode="det")
        assert np.array_equal(p.idx, ref.idx)
        assert np.array_equal(p.val, ref.val)
        assert_trace_equal(ctx.trace(), ref.trace)
        assert (st.rounds, st.pushes, st.pushed_edges) == (ref.rounds, ref.pushes,
                                                            ref.pushed_edges)


@pytest.mark.parametrize("name,t,N,eps", HK_CASES)
def test_hkpr_atomic_within_tolerance(ctx, form, name, t, N, eps):
    off, col, g = gpu_graph(ctx, name)
    for x in seeds_for(off, col, 2, salt=2):
        ref = oracle.hkpr(off, col, x, t, N, eps)
        p, st = lgc.hkpr(g, x, t, N, eps, mode="atomic")
        assert rel_l1(p.idx, p.val, ref.idx, ref.val) <= ATOL_REL_L1


@pytest.mark.parametrize("name,t,N,eps", [("rmat10", 5.0, 12, 1e-2), ("rmat13", 3.0, 10, 1e-3),
                                          ("paper", 1.0, 2, 1.0)])
def test_hkpr_threshold_sign_debug_flag(ctx, name, t, N, eps):
    """LGC_OPT_HK_THRESHOLD_SIGN = -1 (Sec. 3.4's sequential e^{-t} in the
    entry thresholds): the GPU matches the oracle's same reading, bit for bit
    in deterministic mode, and the flag does change the result."""
    off, col, g = gpu_graph(ctx, name)
    x = seeds_for(off, col, 1)[0]
    ctx.set_option(lgc.OPT_HK_THRESHOLD_SIGN, -1)
    try:
        ref = oracle.hkpr(off, col, x, t, N, eps, trace=True, threshold_sign=-1)
        p, st = lgc.hkpr(g, x, t, N, eps, mode="det")
        assert np.array_equal(p.idx, ref.idx) and np.array_equal(p.val, ref.val)
        assert_trace_equal(ctx.trace(), ref.trace)
        assert st.pushed_edges == ref.pushed_edges
        p, st = lgc.hkpr(g, x, t, N, eps, mode="atomic")
        assert rel_l1(p.idx, p.val, ref.idx, ref.val) <= ATOL_REL_L1
    finally:
        ctx.set_option(lgc.OPT_HK_THRESHOLD_SIGN, 1)
    plus = oracle.hkpr(off, col, x, t, N, eps)
    assert plus.pushed_edges < ref.pushed_edges
    p, st = lgc.hkpr(g, x, t, N, eps, mode="det")
    assert np.array_equal(p.val, plus.val) and st.pushed_edges == plus.pushed_edges


# ---------------------------------------------------------------------------
# rand-HK-PR
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("name,t,K,walks", [("paper", 2.0, 5, 10000), ("rmat13", 10.0, 10, 300001),
                                            ("grid6", 3.0, 0, 999), ("rmat16", 10.0, 10, 100000)])
def test_rand_hkpr_bitexact(ctx, name, t, K, walks):
    off, col, g = gpu_graph(ctx, name)
    x = inputs.config1_seed(off, col)
    ref = oracle.rand_hkpr(off, col, x, t, K, walks, 7)
    p, st = lgc.rand_hkpr(g, x, t, K, walks, 7)
    assert np.array_equal(ctx.rand_hkpr_endpoints(walks), ref.endpoints)
    assert np.array_equal(p.idx, ref.idx) and np.array_equal(p.val, ref.val)
    assert st.pushed_edges == ref.pushed_edges


# ---------------------------------------------------------------------------
# graph validation
# ---------------------------------------------------------------------------
def test_graph_validation_rejects_bad_csr(ctx):
    bad = [
        (np.array([0, 1, 1], np.int64), np.array([1], np.int32)),        # asymmetric
        (np.array([0, 1, 2], np.int64), np.array([0, 1], np.int32)),     # self loops
        (np.array([0, 2, 3, 4], np.int64), np.array([2, 1, 0, 0], np.int32)),  # unsorted
        (np.array([0, 2, 3], np.int64), np.array([1, 1, 0], np.int32)),  # duplicate
    ]
    for off, col in bad:
        with pytest.raises(lgc.LgcError):
            lgc.Graph(ctx, off, col, validate=True)


# ---------------------------------------------------------------------------
# deterministic pull rounds (every vertex gathers from its in-frontier
# neighbours in ascending id): forced on every round, they must still be
# bit-identical to the oracle
# ---------------------------------------------------------------------------
OPT_PULL = 7


@pytest.mark.parametrize("name", ["paper", "star40", "grid6", "rand500", "rmat10", "rmat13"])
def test_det_pull_rounds_bitexact(ctx, name):
    off, col, g = gpu_graph(ctx, name)
    ctx.set_option(OPT_PULL, 2)
    try:
        for x in seeds_for(off, col, 2, salt=3):
            for rule in ("opt", "orig"):
                ref = oracle.prnibble(off, col, x, 0.05, 1e-5, rule=1 if rule == "orig" else 0,
                                      trace=True)
                p, st = lgc.prnibble(g, x, 0.05, 1e-5, rule=rule, mode="det")
                assert np.array_equal(p.idx, ref.idx) and np.array_equal(p.val, ref.val)
                r = ctx.residual()
                assert np.array_equal(r.idx, ref.idx2) and np.array_equal(r.val, ref.val2)
                assert_trace_equal(ctx.trace(), ref.trace)
            ref = oracle.nibble(off, col, x, 10, 1e-4, trace=True)
            p, st = lgc.nibble(g, x, 10, 1e-4, mode="det")
            assert np.array_equal(p.idx, ref.idx) and np.array_equal(p.val, ref.val)
            assert_trace_equal(ctx.trace(), ref.trace)
            for t, N, eps in [(5.0, 12, 1e-4), (3.0, 5, 0.0)]:
                ref = oracle.hkpr(off, col, x, t, N, eps, trace=True)
                p, st = lgc.hkpr(g, x, t, N, eps, mode="det")
                assert np.array_equal(p.idx, ref.idx) and np.array_equal(p.val, ref.val)
                assert_trace_equal(ctx.trace(), ref.trace)
    finally:
        ctx.set_option(OPT_PULL, 0)


@pytest.mark.parametrize("name", ["paper", "star40", "grid6", "rand500", "rmat10", "rmat13"])
def test_atomic_pull_rounds_within_tolerance(ctx, name):
    """Atomic mode with every round gathering (heavy vertices reduced by a
    warp butterfly, so the order of additions differs from the oracle's)."""
    off, col, g = gpu_graph(ctx, name)
    ctx.set_option(OPT_PULL, 2)
    try:
        for x in seeds_for(off, col, 2, salt=4):
            ref = oracle.prnibble(off, col, x, 0.05, 1e-5, trace=True)
            p, st = lgc.prnibble(g, x, 0.05, 1e-5, mode="atomic")
            assert rel_l1(p.idx, p.val, ref.idx, ref.val) <= ATOL_REL_L1
            assert [f.tolist() for f in ctx.trace()] == [f.tolist() for f in ref.trace]
            ref = oracle.nibble(off, col, x, 10, 1e-4)
            p, st = lgc.nibble(g, x, 10, 1e-4, mode="atomic")
            assert rel_l1(p.idx, p.val, ref.idx, ref.val) <= ATOL_REL_L1
            ref = oracle.hkpr(off, col, x, 5.0, 12, 1e-4)
            p, st = lgc.hkpr(g, x, 5.0, 12, 1e-4, mode="atomic")
            assert rel_l1(p.idx, p.val, ref.idx, ref.val) <= ATOL_REL_L1
    finally:
        ctx.set_option(OPT_PULL, 0)


# ---------------------------------------------------------------------------
# Device-driven rounds (consecutive small atomic PR-Nibble rounds in one
# cooperative launch): same rounds, pushes and p as the host-driven rounds
# and the oracle.  Tracing is off here (it keeps rounds on the host).
# ---------------------------------------------------------------------------
@pytest.fixture(scope="module")
def ctx_notrace():
    c = lgc.Context(0)
    yield c
    c.close()


DEV_CASES = [("paper", 0.1, 1e-4), ("star40", 0.05, 1e-4), ("grid6", 0.05, 1e-5),
             ("rand500", 0.01, 1e-6), ("rmat10", 0.01, 1e-6), ("rmat13", 0.05, 1e-7),
             ("rmat16", 0.01, 1e-7), ("rmat16", 0.01, 1e-5)]


@pytest.mark.parametrize("rule", ["opt", "orig"])
@pytest.mark.parametrize("form_", [0, 1, 2], ids=["auto", "hashed", "dense"])
@pytest.mark.parametrize("name,alpha,eps", DEV_CASES)
def test_prnibble_device_rounds(ctx_notrace, name, alpha, eps, form_, rule):
    c = ctx_notrace
    off, col = GRAPHS[name]()
    g = lgc.Graph(c, off, col)
    c.set_option(lgc.OPT_TABLE_FORM, form_)
    try:
        for x in seeds_for(off, col, 3, salt=7):
            ref = oracle.prnibble(off, col, x, alpha, eps, rule=0 if rule == "opt" else 1)
            c.set_option(lgc.OPT_DEVICE_ROUNDS, 1)
            p1, s1 = lgc.prnibble(g, x, alpha, eps, rule=rule, mode="atomic")
            c.set_option(lgc.OPT_DEVICE_ROUNDS, 0)
            p0, s0 = lgc.prnibble(g, x, alpha, eps, rule=rule, mode="atomic")
            for p, s in ((p1, s1), (p0, s0)):
                assert (s.rounds, s.pushes, s.pushed_edges) == (ref.rounds, ref.pushes,
                                                                 ref.pushed_edges)
                assert rel_l1(p.idx, p.val, ref.idx, ref.val) <= ATOL_REL_L1
    finally:
        c.set_option(lgc.OPT_DEVICE_ROUNDS, 1)
        c.set_option(lgc.OPT_TABLE_FORM, 0)
        g.close()


def test_prnibble_device_rounds_round_limit(ctx_notrace):
    c = ctx_notrace
    off, col = GRAPHS["rmat13"]()
    g = lgc.Graph(c, off, col)
    try:
        x = inputs.config1_seed(off, col)
        for k in (1, 2, 5):
            ref = oracle.prnibble(off, col, x, 0.01, 1e-6, max_rounds=k)
            p, st = lgc.prnibble(g, x, 0.01, 1e-6, mode="atomic", max_rounds=k)
            assert st.rounds == k and st.pushed_edges == ref.pushed_edges
            assert rel_l1(p.idx, p.val, ref.idx, ref.val) <= ATOL_REL_L1
    finally:
        g.close()


NIB_DEV_CASES = [("paper", 4, 1e-3), ("path9", 10, 0.3), ("star40", 6, 1e-4),
                 ("grid6", 12, 1e-5), ("rand500", 15, 1e-6), ("rmat10", 20, 1e-6),
                 ("rmat13", 20, 1e-7), ("rmat13", 4, 0.0), ("rmat16", 20, 1e-7),
                 ("rmat16", 30, 1e-6)]


@pytest.mark.parametrize("form_", [0, 1, 2], ids=["auto", "hashed", "dense"])
@pytest.mark.parametrize("name,T,eps", NIB_DEV_CASES)
def test_nibble_device_rounds(ctx_notrace, name, T, eps, form_):
    """Nibble's device-driven rounds (atomic mode, tracing off): the same
    rounds, pushes and p as the host-driven rounds and the oracle, including
    runs that end on an empty frontier (the previous p is returned) and runs
    cut by T."""
    c = ctx_notrace
    off, col = GRAPHS[name]()
    g = lgc.Graph(c, off, col)
    c.set_option(lgc.OPT_TABLE_FORM, form_)
    try:
        for x in seeds_for(off, col, 3, salt=11):
            ref = oracle.nibble(off, col, x, T, eps)
            c.set_option(lgc.OPT_DEVICE_ROUNDS, 1)
            p1, s1 = lgc.nibble(g, x, T, eps, mode="atomic")
            c.set_option(lgc.OPT_DEVICE_ROUNDS, 0)
            p0, s0 = lgc.nibble(g, x, T, eps, mode="atomic")
            for p, s in ((p1, s1), (p0, s0)):
                assert (s.rounds, s.pushes, s.pushed_edges) == (ref.rounds, ref.pushes,
                                                                 ref.pushed_edges)
                assert rel_l1(p.idx, p.val, ref.idx, ref.val) <= ATOL_REL_L1
    finally:
        c.set_option(lgc.OPT_DEVICE_ROUNDS, 1)
        c.set_option(lgc.OPT_TABLE_FORM, 0)
        g.close()


# ---------------------------------------------------------------------------
# Heavy-vertex pull gather: every batch depth gives the same (exact) sums, and
# the autotuner picks one of them.
# ---------------------------------------------------------------------------
def test_pull_batch_depths_bit_identical(ctx_notrace):
    c = ctx_notrace
    off, col = GRAPHS["rmat16"]()
    g = lgc.Graph(c, off, col)
    c.set_option(lgc.OPT_DEVICE_ROUNDS, 0)
    c.set_option(lgc.OPT_PULL, 2)  # every round a pull round: no atomics decide the order
    try:
        x = inputs.config1_seed(off, col)
        ref = oracle.prnibble(off, col, x, 0.01, 1e-6)
        res = []
        shapes = [(b, gw, sb) for sb in (16, 8)
                  for b, gw in ((4, 32), (8, 32), (16, 32), (8, 16), (16, 16), (8, 8), (16, 8))]
        for b, gw, sb in shapes:
            c.set_option(lgc.OPT_PULL_BATCH, b)
            c.set_option(lgc.OPT_PULL_GROUP, gw)
            c.set_option(lgc.OPT_PULL_SHARE, sb)
            p, st = lgc.prnibble(g, x, 0.01, 1e-6, mode="atomic")
            assert (st.rounds, st.pushed_edges) == (ref.rounds, ref.pushed_edges)
            assert rel_l1(p.idx, p.val, ref.idx, ref.val) <= ATOL_REL_L1
            res.append(p)
        for p in res[1:]:
            assert np.array_equal(p.idx, res[0].idx) and np.array_equal(p.val, res[0].val)
        c.set_option(lgc.OPT_PULL_BATCH, 0)
        c.set_option(lgc.OPT_PULL_GROUP, 0)
        c.set_option(lgc.OPT_PULL_SHARE, 0)
        assert g.pull_light() == 32  # the default degree bin
        default_handoff = g.batch_handoff()
        assert default_handoff == max(1 << 20, g.nnz // 64)
        assert g.autotune() in shapes
        p, st = lgc.prnibble(g, x, 0.01, 1e-6, mode="atomic")
        assert np.array_equal(p.idx, res[0].idx) and np.array_equal(p.val, res[0].val)
        assert g.pull_light() in (32, 64, 128, 256)
        # the batch hand-off threshold is one of the tuner's candidates
        assert g.batch_handoff() in {max(1 << 20, g.nnz // k) for k in (64, 16, 4)} | {2 ** 63 - 1}
        ps, sts = lgc.prnibble_batch(g, [x, int(col[0])], 0.01, 1e-6, mode="det")
        ref2 = oracle.prnibble(off, col, int(col[0]), 0.01, 1e-6)
        assert np.array_equal(ps[0].idx, ref.idx) and np.array_equal(ps[0].val, ref.val)
        assert np.array_equal(ps[1].idx, ref2.idx) and np.array_equal(ps[1].val, ref2.val)
    finally:
        c.set_option(lgc.OPT_PULL_BATCH, 0)
        c.set_option(lgc.OPT_PULL_GROUP, 0)
        c.set_option(lgc.OPT_PULL_SHARE, 0)
        c.set_option(lgc.OPT_PULL, 0)
        c.set_option(lgc.OPT_DEVICE_ROUNDS, 1)
        g.close()


@pytest.mark.parametrize("light", [4, 16, 64, 256])
def test_pull_degree_bins(ctx, light):
    """The atomic pull rounds' degree bin (vertices of degree <= light gather
    one thread each; deterministic mode keeps its own bins at any light: one
    thread each up to degree 32, one lane each up to 1024, then
    segment-parallel; the sweep of a large support walks the same lists)
    changes speed only: HK-PR's
    near-global pull rounds and PR-Nibble with every round a pull round give
    the oracle's results, bit for bit in deterministic mode."""
    off, col = inputs.rmat(16, seed=1)
    g = lgc.Graph(ctx, off, col)
    x = inputs.config1_seed(off, col)
    try:
        g.set_pull_light(light)
        assert g.pull_light() == light
        ref = oracle.hkpr(off, col, x, 10.0, 20, 1e-7, trace=True)
        p, st = lgc.hkpr(g, x, 10.0, 20, 1e-7, mode="det")
        assert np.array_equal(p.idx, ref.idx) and np.array_equal(p.val, ref.val)
        assert_trace_equal(ctx.trace(), ref.trace)
        # the sweep of a support over n/32 walks the same degree-binned lists
        assert len(p.idx) >= (len(off) - 1) // 32
        rs = oracle.sweep(off, col, ref.idx, ref.val)
        c = lgc.sweep(g, p)
        assert (c.size, c.vol, c.cut) == (rs.best, rs.best_vol, rs.best_cut)
        assert np.array_equal(c.ids, rs.cluster) and c.conductance == rs.conductance
        p, st = lgc.hkpr(g, x, 10.0, 20, 1e-7, mode="atomic")
        assert rel_l1(p.idx, p.val, ref.idx, ref.val) <= ATOL_REL_L1
        ctx.set_option(lgc.OPT_PULL, 2)
        ref = oracle.prnibble(off, col, x, 0.01, 1e-6)
        for mode in ("det", "atomic"):
            p, st = lgc.prnibble(g, x, 0.01, 1e-6, mode=mode)
            assert st.pushed_edges == ref.pushed_edges
            if mode == "det":
                assert np.array_equal(p.idx, ref.idx) and np.array_equal(p.val, ref.val)
            else:
                assert rel_l1(p.idx, p.val, ref.idx, ref.val) <= ATOL_REL_L1
    finally:
        ctx.set_option(lgc.OPT_PULL, 0)
        g.close()
    with pytest.raises(lgc.LgcError):
        g2 = lgc.Graph(ctx, off, col)
        try:
            g2.set_pull_light(3)
        finally:
            g2.close()
