"""Pins for the CPU oracle: checks against facts the paper and the mathematics
fix, independent of the oracle's own code (dense linear algebra, closed
forms, the paper's worked example, brute force, hand-worked traces)."""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_1604_07515_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def small_graphs():
    yield "paper", inputs.paper_example(), 2
    yield "path7", inputs.path(7), 3
    yield "star6", inputs.star(6), 0
    yield "cliques4", inputs.clique_pair(4), 1
    yield "grid3", inputs.grid3d(3), 5
    yield "rand30", inputs.random_graph(30, 70, seed=11), 4


def dense(off, col):
    n = len(off) - 1
    A = np.zeros((n, n))
    for v in range(n):
        A[v, col[off[v]:off[v + 1]]] = 1.0
    d = A.sum(axis=0)
    return A, d


def walk_matrix(off, col):
    """P = A D^-1 (column stochastic) and the lazy walk W = (I + P)/2."""
    A, d = dense(off, col)
    with np.errstate(divide="ignore"):
        Dinv = np.diag(np.where(d > 0, 1.0 / d, 0.0))
    P = A @ Dinv
    return P, 0.5 * (np.eye(len(d)) + P), d


def to_dense(n, idx, val):
    x = np.zeros(n)
    x[idx] = val
    return x


# ---------------------------------------------------------------------------
# Sweep cut (Sec. 3.1, Theorem thm:sweep)
# ---------------------------------------------------------------------------
def test_sweep_worked_example_matches_paper():
    g = json.load(open(os.path.join(GOLDEN, "sweep_worked_example.json")))
    off, col = inputs.paper_example()
    # any p with p/d non-increasing in the order A, B, C, D
    p = np.array([0.4, 0.3, 0.3, 0.2])
    res = oracle.sweep(off, col, np.arange(4), p)
    assert res.order.tolist() == [0, 1, 2, 3]
    assert np.diff(off)[:4].tolist() == g["degrees"]
    assert res.vol.tolist() == g["volumes"]
    assert res.cut.tolist() == g["crossing_edges"]
    assert res.best == len(g["answer"])
    assert res.conductance == 1.0 / 7.0
    z = oracle.sweep_zpath(off, col, res.order)
    assert z.z.tolist() == g["Z"]
    assert z.z_sorted.tolist() == g["Z_sorted"]
    assert z.z_summed.tolist() == g["Z_sorted_summed"]
    assert z.cut.tolist() == g["crossing_edges"]
    assert z.vol.tolist() == g["volumes"]


def brute_force_sweep(off, col, idx, val):
    """Every prefix enumerated; boundary counted edge by edge."""
    d = np.diff(off)
    keep = val > 0
    idx, val = idx[keep], val[keep]
    key = val / d[idx]
    order = idx[np.lexsort((idx, -key))]
    n, two_m = len(d), int(off[-1])
    src = np.repeat(np.arange(n), d)
    best, best_phi, vols, cuts = 0, None, [], []
    for i in range(1, len(order) + 1):
        inS = np.zeros(n, bool)
        inS[order[:i]] = True
        cut = int(np.sum(inS[src] & ~inS[col]))
        vol = int(d[order[:i]].sum())
        vols.append(vol)
        cuts.append(cut)
        den = min(vol, two_m - vol)
        if den > 0:
            phi = Fraction(cut, den)
            if best_phi is None or phi < best_phi:
                best, best_phi = i, phi
    return order, vols, cuts, best, best_phi


@pytest.mark.parametrize("name,g,seed", list(small_graphs()))
def test_sweep_brute_force(name, g, seed):
    off, col = g
    n = len(off) - 1
    rng = np.random.default_rng(seed + 100)
    for trial in range(5):
        k = rng.integers(1, n + 1)
        idx = np.sort(rng.choice(n, size=k, replace=False))
        idx = idx[np.diff(off)[idx] > 0]
        # values on a coarse grid so that p/d ties occur
        val = rng.integers(0, 4, size=len(idx)) * 0.25 * np.diff(off)[idx]
        res = oracle.sweep(off, col, idx, val)
        order, vols, cuts, best, phi = brute_force_sweep(off, col, idx, val)
        assert res.order.tolist() == order.tolist()
        assert res.vol.tolist() == vols
        assert res.cut.tolist() == cuts
        assert res.best == best
        if best:
            assert Fraction(res.best_cut, min(res.best_vol, int(off[-1]) - res.best_vol)) == phi
        z = oracle.sweep_zpath(off, col, res.order)
        assert z.cut.tolist() == cuts


def test_sweep_empty_and_global():
    off, col = inputs.paper_example()
    res = oracle.sweep(off, col, np.zeros(0, np.int32), np.zeros(0))
    assert res.best == 0 and math.isinf(res.conductance)
    # whole graph: the last prefix has denominator 0 and is skipped
    n = len(off) - 1
    res = oracle.sweep(off, col, np.arange(n), np.ones(n))
    assert res.vol[-1] == off[-1] and res.cut[-1] == 0
    assert res.best < n


# ---------------------------------------------------------------------------
# PR-Nibble (Sec. 3.3)
# ---------------------------------------------------------------------------
def ppr(W, alpha, s):
    """pr_alpha(s) = alpha (I - (1 - alpha) W)^-1 s (Andersen-Chung-Lang)."""
    n = len(s)
    return alpha * np.linalg.solve(np.eye(n) - (1.0 - alpha) * W, s)


@pytest.mark.parametrize("rule", [0, 1])
@pytest.mark.parametrize("name,g,seed", list(small_graphs()))
def test_prnibble_invariant_every_round(name, g, seed, rule):
    off, col = g
    n = len(off) - 1
    P, W, d = walk_matrix(off, col)
    alpha, eps = 0.15, 1e-4
    chi = np.zeros(n)
    chi[seed] = 1.0
    pstar = ppr(W, alpha, chi)
    full = oracle.prnibble(off, col, seed, alpha, eps, rule=rule)
    assert full.status == 0
    for k in range(1, full.rounds + 1):
        res = oracle.prnibble(off, col, seed, alpha, eps, rule=rule, max_rounds=k)
        p = to_dense(n, res.idx, res.val)
        r = to_dense(n, res.idx2, res.val2)
        assert np.abs(p + ppr(W, alpha, r) - pstar).max() < 1e-13
        assert abs(p.sum() + r.sum() - 1.0) < 1e-14
        assert r.min() >= 0.0
    p = to_dense(n, full.idx, full.val)
    r = to_dense(n, full.idx2, full.val2)
    gap = pstar - p
    assert gap.min() > -1e-14 and np.all(gap <= eps * d + 1e-14)
    assert np.all(r < eps * d)
    assert full.pushed_edges <= 1.0 / (alpha * eps)


def test_prnibble_hand_worked_two_vertices():
    """Single edge 0-1, seed 0, alpha = 1/2 (so 2a/(1+a) = 2/3 and
    (1-a)/(1+a) = 1/3), eps = 0.02, optimized rule, traced by hand:
      round 1: F={0}: p0 = 2/3,          r0 = 0, r1 = 1/3
      round 2: F={1}: p1 = 2/9,          r1 = 0, r0 = 1/9
      round 3: F={0}: p0 = 2/3 + 2/27,   r0 = 0, r1 = 1/27
      round 4: F={1}: p1 = 2/9 + 2/81,   r1 = 0, r0 = 1/81 < 0.02: stop."""
    off, col = inputs.path(2)
    res = oracle.prnibble(off, col, 0, 0.5, 0.02, rule=0, trace=True)
    assert res.rounds == 4
    assert [f.tolist() for f in res.trace] == [[0], [1], [0], [1]]
    np.testing.assert_allclose(res.val, [2 / 3 + 2 / 27, 2 / 9 + 2 / 81], rtol=0, atol=1e-16)
    np.testing.assert_allclose(res.val2, [1 / 81, 0.0], rtol=0, atol=1e-17)


def test_prnibble_hand_worked_star_original_rule():
    """Star with centre 0 and 4 leaves, seed 0, alpha = 1/2, original rule,
    eps = 0.1.  Round 1: F={0}: p0 = 1/2, r0 = (1/2)(1)/2 = 1/4, each leaf
    r = (1/2)/(2*4) = 1/16.  Thresholds: centre 0.4, leaf 0.1: nobody
    qualifies, so one round."""
    off, col = inputs.star(4)
    res = oracle.prnibble(off, col, 0, 0.5, 0.1, rule=1, trace=True)
    assert res.rounds == 1
    assert res.idx.tolist() == [0] and res.val.tolist() == [0.5]
    assert res.idx2.tolist() == [0, 1, 2, 3, 4]
    assert res.val2.tolist() == [0.25, 1 / 16, 1 / 16, 1 / 16, 1 / 16]
    # eps = 0.05: the leaves qualify (1/16 >= 0.05) and so does the centre
    # (1/4 >= 0.05 * 4), all in round 2
    res = oracle.prnibble(off, col, 0, 0.5, 0.05, rule=1, trace=True)
    assert [f.tolist() for f in res.trace][:2] == [[0], [0, 1, 2, 3, 4]]


def test_prnibble_both_rules_same_system():
    """Sec. 3.3: both rules approximate the same PPR vector."""
    off, col = inputs.clique_pair(5)
    n = len(off) - 1
    _, W, d = walk_matrix(off, col)
    chi = np.zeros(n)
    chi[2] = 1.0
    pstar = ppr(W, 0.1, chi)
    for rule in (0, 1):
        res = oracle.prnibble(off, col, 2, 0.1, 1e-9, rule=rule)
        assert np.abs(to_dense(n, res.idx, res.val) - pstar).max() < 1e-7


# PR-Nibble from a seed set, beta-fraction rounds (Sec. 3 seed sets; Sec. 3.3
# beta variant).  Pins: the dense PPR invariant with the seed distribution
# after every round, the terminal guarantee, the work bound, and the
# hand-worked order of a star.
@pytest.mark.parametrize("beta", [1.0, 0.5, 0.2, 1e-9])
@pytest.mark.parametrize("rule", [0, 1])
def test_prnibble_set_invariant_every_round(beta, rule):
    off, col = inputs.random_graph(60, 200, seed=4)
    n = len(off) - 1
    _, W, d = walk_matrix(off, col)
    cand = np.flatnonzero(d > 0)
    seeds = cand[[0, 5, 9]].astype(np.int32)
    w = np.array([1.0, 2.0, 0.5])
    s = np.zeros(n)
    Wsum = (1.0 + 2.0) + 0.5
    s[seeds] = w / Wsum
    pstar = ppr(W, 0.1, s)
    eps = 1e-4
    full = oracle.prnibble_set(off, col, seeds, w, 0.1, eps, rule=rule, beta=beta, trace=True)
    assert full.status == 0
    for k in range(1, min(full.rounds, 40) + 1):
        res = oracle.prnibble_set(off, col, seeds, w, 0.1, eps, rule=rule, beta=beta, max_rounds=k)
        p = to_dense(n, res.idx, res.val)
        r = to_dense(n, res.idx2, res.val2)
        assert np.abs(p + ppr(W, 0.1, r) - pstar).max() < 1e-13
        assert abs(p.sum() + r.sum() - 1.0) < 1e-14
    p = to_dense(n, full.idx, full.val)
    r = to_dense(n, full.idx2, full.val2)
    gap = pstar - p
    assert gap.min() > -1e-14 and np.all(gap <= eps * d + 1e-14)
    assert np.all(r < eps * d)
    assert full.pushed_edges <= 1.0 / (0.1 * eps)
    if beta == 1e-9:  # one vertex per round
        assert all(len(f) == 1 for f in full.trace) and full.pushes == full.rounds


def test_prnibble_set_one_seed_is_prnibble():
    off, col = inputs.rmat(10, seed=5)
    x = inputs.config1_seed(off, col)
    a = oracle.prnibble(off, col, x, 0.05, 1e-5)
    b = oracle.prnibble_set(off, col, [x], [1.0], 0.05, 1e-5)
    assert np.array_equal(a.idx, b.idx) and np.array_equal(a.val, b.val)
    assert (a.rounds, a.pushes, a.pushed_edges) == (b.rounds, b.pushes, b.pushed_edges)


def test_prnibble_set_beta_hand_worked_star():
    """Star, centre 0 and leaves 1..4, seeds {1, 2} with weights 3 and 1
    (r = 3/4, 1/4), alpha = 1/2 (optimized rule: 2a/(1+a) = 2/3,
    (1-a)/(1+a) = 1/3), eps = 0.01, beta = 0.5: both seeds qualify
    (r/d = 3/4 and 1/4); ceil(0.5 * 2) = 1 pushes, the larger r/d: leaf 1.
    Round 1: p1 = 1/2, r1 = 0, r0 = 1/4; frontier {0, 2} (1/4 >= 0.04)."""
    off, col = inputs.star(4)
    res = oracle.prnibble_set(off, col, [1, 2], [3.0, 1.0], 0.5, 0.01, beta=0.5,
                              max_rounds=1, trace=True)
    assert [f.tolist() for f in res.trace] == [[1]]
    assert res.idx.tolist() == [1] and res.val.tolist() == [0.5]
    assert res.idx2.tolist() == [0, 1, 2] and res.val2.tolist() == [0.25, 0.0, 0.25]
    # round 2: r/d of 0 is (1/4)/4 = 1/16, of leaf 2 is 1/4: leaf 2 pushes
    res = oracle.prnibble_set(off, col, [1, 2], [3.0, 1.0], 0.5, 0.01, beta=0.5,
                              max_rounds=2, trace=True)
    assert [f.tolist() for f in res.trace] == [[1], [2]]


def test_prnibble_set_rejects_bad_sets():
    off, col = inputs.star(4)
    for seeds, w, beta in [([1, 1], [1.0, 1.0], 1.0), ([1], [0.0], 1.0), ([1], [1.0], 0.0),
                           ([1], [1.0], 1.5), ([9], [1.0], 1.0)]:
        assert oracle.prnibble_set(off, col, seeds, w, 0.1, 1e-3, beta=beta).status == -1


def test_prnibble_queue_vs_synchronous():
    """The sequential queue version reaches the same accuracy guarantee; the
    synchronous version does at least roughly as many pushes (Table
    table:pr-nibble reports 1.0-1.6x)."""
    off, col = inputs.rmat(10, seed=5)
    n = len(off) - 1
    d = np.diff(off)
    x = inputs.config1_seed(off, col)
    _, W, _ = walk_matrix(off, col)
    chi = np.zeros(n)
    chi[x] = 1.0
    pstar = ppr(W, 0.05, chi)
    eps = 1e-5
    for res in (oracle.prnibble(off, col, x, 0.05, eps), oracle.prnibble_queue(off, col, x, 0.05, eps)):
        gap = pstar - to_dense(n, res.idx, res.val)
        assert gap.min() > -1e-13 and np.all(gap <= eps * d + 1e-13)


# ---------------------------------------------------------------------------
# Nibble (Sec. 3.2)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("name,g,seed", list(small_graphs()))
def test_nibble_eps0_is_lazy_walk(name, g, seed):
    off, col = g
    n = len(off) - 1
    _, W, _ = walk_matrix(off, col)
    x = np.zeros(n)
    x[seed] = 1.0
    for T in range(0, 6):
        res = oracle.nibble(off, col, seed, T, 0.0)
        p = to_dense(n, res.idx, res.val)
        assert np.abs(p - x).max() < 1e-14
        assert abs(p.sum() - 1.0) < 1e-14
        x = W @ x


def test_nibble_early_exit_hand_worked():
    """Path 0-1-2, seed 0, eps = 0.3.  t=1: p' = {0: 1/2, 1: 1/2}; vertex 0
    (d=1) passes 1/2 >= 0.3, vertex 1 (d=2) fails 1/2 < 0.6: F = {0}, p = p'.
    t=2: p' = {0: 1/4, 1: 1/4}: nobody passes, so p_1 is returned."""
    off, col = inputs.path(3)
    res = oracle.nibble(off, col, 0, 10, 0.3, trace=True)
    assert res.idx.tolist() == [0, 1] and res.val.tolist() == [0.5, 0.5]
    assert res.rounds == 2
    assert [f.tolist() for f in res.trace] == [[0], [0]]


def test_nibble_truncation_mass():
    """Each step keeps exactly the frontier's mass: sum p_T = sum_{v in F_T}
    p_{T-1}(v).  A run of T steps returns p_T while the frontier after step T
    is non-empty (F_{T+1} exists in the trace of a longer run)."""
    off, col = inputs.rmat(9, seed=3)
    x = inputs.config1_seed(off, col)
    longest = oracle.nibble(off, col, x, 50, 1e-3, trace=True)
    R = len(longest.trace)
    assert 3 <= R < 50
    prev = oracle.nibble(off, col, x, 1, 1e-3)
    for T in range(2, R):
        res = oracle.nibble(off, col, x, T, 1e-3)
        F = longest.trace[T - 1]
        pv = dict(zip(prev.idx.tolist(), prev.val.tolist()))
        assert abs(res.val.sum() - sum(pv[v] for v in F.tolist())) < 1e-14
        prev = res
    # after the last non-empty frontier the run returns the previous vector
    tail = oracle.nibble(off, col, x, R + 5, 1e-3)
    assert tail.idx.tolist() == prev.idx.tolist() and tail.val.tolist() == prev.val.tolist()


# ---------------------------------------------------------------------------
# HK-PR (Sec. 3.4)
# ---------------------------------------------------------------------------
def test_hkpr_psi_recurrence_equals_sum():
    for t, N in [(1.0, 5), (3.0, 10), (10.0, 20), (30.0, 60)]:
        psi = oracle.hkpr_psi(t, N)
        for k in range(N + 1):
            exact = sum(Fraction(math.factorial(k), math.factorial(m + k)) * Fraction(t) ** m
                        for m in range(N - k + 1))
            assert abs(psi[k] - float(exact)) <= 1e-14 * float(exact)


@pytest.mark.parametrize("name,g,seed", list(small_graphs()))
def test_hkpr_eps0_closed_form(name, g, seed):
    """With eps = 0 every touched vertex stays on the frontier and p equals
    sum_{k<N} t^k/k! P^k chi + t^(N-1)/(N-1)! P^N chi (the last level adds
    r/d without a t/N factor, Fig. alg:hkpr)."""
    off, col = g
    n = len(off) - 1
    P, _, _ = walk_matrix(off, col)
    for t, N in [(1.5, 4), (3.0, 7)]:
        chi = np.zeros(n)
        chi[seed] = 1.0
        expect = np.zeros(n)
        v = chi.copy()
        for k in range(N):
            expect += (t ** k / math.factorial(k)) * v
            v = P @ v
        expect += (t ** (N - 1) / math.factorial(N - 1)) * v
        res = oracle.hkpr(off, col, seed, t, N, 0.0)
        p = to_dense(n, res.idx, res.val)
        assert np.abs(p - expect).max() <= 1e-13 * expect.max()
        assert res.rounds == N


@pytest.mark.parametrize("eps", [1e-3, 1e-4])
def test_hkpr_queue_equals_levels(eps):
    """Sec. 3.4: the level-synchronous version applies the same updates as the
    sequential queue version (same support; values equal up to order)."""
    off, col = inputs.rmat(10, seed=7)
    x = inputs.config1_seed(off, col)
    a = oracle.hkpr(off, col, x, 5.0, 12, eps)
    b = oracle.hkpr_queue(off, col, x, 5.0, 12, eps)
    assert a.idx.tolist() == b.idx.tolist()
    np.testing.assert_allclose(a.val, b.val, rtol=1e-13, atol=0)


def test_hkpr_hand_worked_threshold():
    """Star with centre 0 and 3 leaves, seed 0, t = 1, N = 2.  Level 0:
    p0 += 1; each leaf gets t*1/(1*3) = 1/3.  c_1 = e*eps/(2*2*psi_1) with
    psi_1 = 1 + t/2 = 1.5.  For eps = 1 the leaf threshold is e/6 = 0.453 >
    1/3: frontier empty, p = {0: 1}.  For eps = 0.5 it is 0.2265 <= 1/3: the
    leaves go on; level 1 is the last: p[leaf] += 1/3, p[0] += 3 * (1/3)/1."""
    off, col = inputs.star(3)
    res = oracle.hkpr(off, col, 0, 1.0, 2, 1.0)
    assert res.idx.tolist() == [0] and res.val.tolist() == [1.0]
    res = oracle.hkpr(off, col, 0, 1.0, 2, 0.5)
    assert res.idx.tolist() == [0, 1, 2, 3]
    np.testing.assert_allclose(res.val, [2.0, 1 / 3, 1 / 3, 1 / 3], rtol=1e-15)


def test_hkpr_threshold_sign_hand_worked():
    """The e^{-t} thresholds of Sec. 3.4's sequential description (the
    debug reading; the parallel figure's e^{t} is the default).  Same star,
    t = 1, N = 2: c_1 = e^-1 eps / (2 * 2 * 1.5) = eps / (6e).  eps = 1 gives
    0.0613 <= 1/3, so the leaves go on (with e^{t} they did not); eps = 6
    gives 1/e = 0.368 > 1/3: frontier empty."""
    off, col = inputs.star(3)
    res = oracle.hkpr(off, col, 0, 1.0, 2, 1.0, threshold_sign=-1)
    assert res.idx.tolist() == [0, 1, 2, 3]
    np.testing.assert_allclose(res.val, [2.0, 1 / 3, 1 / 3, 1 / 3], rtol=1e-15)
    res = oracle.hkpr(off, col, 0, 1.0, 2, 6.0, threshold_sign=-1)
    assert res.idx.tolist() == [0] and res.val.tolist() == [1.0]
    a = oracle.hkpr(off, col, 0, 1.0, 2, 0.5)
    b = oracle.hkpr(off, col, 0, 1.0, 2, 0.5, threshold_sign=1)
    assert a.val.tolist() == b.val.tolist()


@pytest.mark.parametrize("t,N,eps", [(3.0, 10, 1e-3), (5.0, 12, 1e-2)])
def test_hkpr_threshold_sign_monotone(t, N, eps):
    """Lower thresholds only add work: with e^{-t} every level's frontier
    contains the e^{t} one and p is pointwise at least as large (each r' is a
    left fold of a superset of larger non-negative terms, and rounding to
    nearest is monotone).  At t >= 3 the e^{-t} run pushes strictly more."""
    off, col = inputs.rmat(10, seed=7)
    n = len(off) - 1
    x = inputs.config1_seed(off, col)
    hi = oracle.hkpr(off, col, x, t, N, eps, trace=True)
    lo = oracle.hkpr(off, col, x, t, N, eps, trace=True, threshold_sign=-1)
    assert len(lo.trace) >= len(hi.trace)
    for f_hi, f_lo in zip(hi.trace, lo.trace):
        assert set(f_hi.tolist()) <= set(f_lo.tolist())
    assert np.all(to_dense(n, lo.idx, lo.val) >= to_dense(n, hi.idx, hi.val))
    assert lo.pushed_edges > hi.pushed_edges


# ---------------------------------------------------------------------------
# rand-HK-PR (Sec. 3.5) and the Philox stream
# ---------------------------------------------------------------------------
def test_rand_hkpr_distribution():
    """E[p] = sum_{k<K} Pois_t(k) P^k chi + P(k >= K) P^K chi."""
    off, col = inputs.paper_example()
    n = len(off) - 1
    P, _, _ = walk_matrix(off, col)
    t, K, walks, seed = 2.0, 5, 200000, 42
    res = oracle.rand_hkpr(off, col, 3, t, K, walks, seed)
    p = to_dense(n, res.idx, res.val)
    chi = np.zeros(n)
    chi[3] = 1.0
    expect = np.zeros(n)
    v = chi.copy()
    tail = 1.0
    for k in range(K):
        pk = math.exp(-t) * t ** k / math.factorial(k)
        expect += pk * v
        tail -= pk
        v = P @ v
    expect += tail * v
    sigma = np.sqrt(expect * (1 - expect) / walks)
    assert np.all(np.abs(p - expect) <= 5 * sigma + 1e-12)
    assert abs(p.sum() - 1.0) < 1e-12
    counts = np.bincount(res.endpoints, minlength=n)
    np.testing.assert_array_equal(to_dense(n, res.idx, res.val), counts / walks)


def test_rand_hkpr_degenerate_lengths():
    off, col = inputs.paper_example()
    res = oracle.rand_hkpr(off, col, 2, 3.0, 0, 1000, 1)   # K = 0: no steps
    assert res.idx.tolist() == [2] and res.val.tolist() == [1.0]
    res = oracle.rand_hkpr(off, col, 2, 3.0, 1, 5000, 1)   # K = 1: 0 or 1 step
    assert set(res.idx.tolist()) <= {0, 1, 2, 3}


def test_philox_uniformity_and_avalanche():
    key = np.array([0x12345678, 0x9ABCDEF0], np.uint32)
    words = np.array([oracle.philox4x32_10([i, 0, 0, 0], key) for i in range(4000)])
    bytes_ = words.view(np.uint8).ravel()
    hist = np.bincount(bytes_, minlength=256)
    e = len(bytes_) / 256
    chi2 = ((hist - e) ** 2 / e).sum()
    assert chi2 < 255 + 6 * math.sqrt(2 * 255)
    bits = np.unpackbits(words.view(np.uint8)).mean()
    assert abs(bits - 0.5) < 0.005
    # one-bit counter change flips about half of the output bits
    flips = []
    for b in range(32):
        a = oracle.philox4x32_10([7, 0, 0, 0], key)
        c = oracle.philox4x32_10([7 ^ (1 << b), 0, 0, 0], key)
        flips.append(np.unpackbits((a ^ c).view(np.uint8)).sum())
    assert 48 < np.mean(flips) < 80
    assert not np.array_equal(oracle.philox4x32_10([1, 2, 3, 4], key),
                              oracle.philox4x32_10([1, 2, 3, 4], key ^ np.uint32(1)))


def _curand_host_philox_blocks(seed, first_block, nblocks):
    """Words of cuRAND's host-side Philox4x32-10 generator (a library routine
    written independently of the oracle), starting at 4-word block
    ``first_block``.  None when libcurand cannot be loaded."""
    import ctypes
    import ctypes.util
    names = ["libcurand.so", "libcurand.so.10"]
    found = ctypes.util.find_library("curand")
    if found:
        names.insert(0, found)
    for root in (os.environ.get("CUDA_HOME"), "/usr/local/cuda"):
        if root:
            names.append(os.path.join(root, "lib64", "libcurand.so"))
    lib = None
    for name in names:
        try:
            lib = ctypes.CDLL(name)
            break
        except OSError:
            continue
    if lib is None:
        return None
    gen = ctypes.c_void_p()
    philox4_32_10 = 161                      # curandRngType_t value in curand.h
    if lib.curandCreateGeneratorHost(ctypes.byref(gen), philox4_32_10) != 0:
        return None
    try:
        assert lib.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
        assert lib.curandSetGeneratorOffset(gen, ctypes.c_ulonglong(4 * first_block)) == 0
        out = np.zeros(4 * nblocks, np.uint32)
        assert lib.curandGenerate(gen, out.ctypes.data_as(ctypes.c_void_p),
                                  ctypes.c_size_t(len(out))) == 0
    finally:
        lib.curandDestroyGenerator(gen)
    return out.reshape(nblocks, 4)


@pytest.mark.parametrize("seed", [0, 0x0123456789ABCDEF, 0xFFFFFFFFFFFFFFFF, 7])
def test_philox_matches_curand_host_generator(seed):
    # cuRAND's host generator keys Philox4x32-10 with the 64-bit seed (low
    # word first) and emits 4-word block b from the counter
    # (b div 2^16 as a 64-bit value in words 0-1, b mod 2^16 in word 2, 0).
    # Blocks near 0, past 2^16 and past 2^48 exercise counter words 0, 1, 2.
    key = np.array([seed & 0xFFFFFFFF, seed >> 32], np.uint32)
    for first in (0, (3 << 16) - 5, (1 << 48) + (9 << 16) + 11):
        got = _curand_host_philox_blocks(seed, first, 32)
        if got is None:
            pytest.skip("libcurand is not available")
        for j in range(32):
            b = first + j
            q, r = b >> 16, b & 0xFFFF
            ctr = [q & 0xFFFFFFFF, q >> 32, r, 0]
            assert np.array_equal(oracle.philox4x32_10(ctr, key), got[j]), (seed, b)
