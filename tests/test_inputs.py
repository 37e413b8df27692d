"""The seeded input generators shared by the oracle and the CUDA path: CSR
invariants of every graph builder, the R-MAT degree profile at scale 16
(n 65,536, about 1.82M directed entries, about 18.8k isolated vertices,
vertex 0 the hub), determinism, and the samplers' ranges."""
import numpy as np
import pytest

from paper_1604_07515_gb300 import inputs


def check_csr(off, col):
    off, col = np.asarray(off), np.asarray(col)
    n = len(off) - 1
    assert off[0] == 0 and off[-1] == len(col)
    assert np.all(np.diff(off) >= 0)
    assert col.dtype == np.int32 and off.dtype == np.int64
    assert len(col) == 0 or (col.min() >= 0 and col.max() < n)
    src = np.repeat(np.arange(n), np.diff(off))
    assert not np.any(src == col)                                  # no self loops
    for v in range(n):                                             # sorted, no duplicates
        assert np.all(np.diff(col[off[v]:off[v + 1]]) > 0)
    fwd = set(zip(src.tolist(), col.tolist()))                     # symmetric
    assert all((w, v) in fwd for v, w in fwd)


@pytest.mark.parametrize("name,g", [
    ("paper", inputs.paper_example()), ("path", inputs.path(9)), ("star", inputs.star(7)),
    ("cliques", inputs.clique_pair(5)), ("grid", inputs.grid3d(4)),
    ("random", inputs.random_graph(60, 200, seed=3)), ("rmat10", inputs.rmat(10, seed=5)),
])
def test_builders_give_valid_csr(name, g):
    check_csr(*g)


def test_small_builders_shapes():
    off, col = inputs.grid3d(4)                   # 3-D torus: degree 6 everywhere
    assert np.all(np.diff(off) == 6)
    off, col = inputs.clique_pair(5)
    assert len(col) == 2 * (2 * 10 + 1)
    off, col = inputs.star(7)
    assert off[1] - off[0] == 7 and np.all(np.diff(off)[1:] == 1)
    off, col = inputs.paper_example()             # n = 8, m = 8; D has degree 4
    assert len(off) == 9 and len(col) == 16 and off[4] - off[3] == 4


def test_rmat_scale16_profile():
    off, col = inputs.rmat(16, seed=1)
    d = np.diff(off)
    assert len(d) == 1 << 16
    assert abs(len(col) - 1.82e6) < 0.05 * 1.82e6
    assert abs((d == 0).sum() - 18.8e3) < 0.15 * 18.8e3
    assert int(d.argmax()) == 0 and 0.7 * 9.7e3 < d.max() < 1.3 * 9.7e3
    assert abs((d >= 2).sum() - 38e3) < 0.1 * 38e3


def test_rmat_is_deterministic_per_seed():
    a = inputs.rmat(11, seed=7, threads=1)
    b = inputs.rmat(11, seed=7, threads=4)
    c = inputs.rmat(11, seed=8)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    assert not (np.array_equal(a[0], c[0]) and np.array_equal(a[1], c[1]))


def test_splitmix_python_and_c_agree():
    lib = inputs._load()
    k = np.array([0, 1, 2, 1000, 123456789, (1 << 40) + 3], np.uint64)
    for seed in (0, 1, 0xDEADBEEF, (1 << 64) - 1):
        py = inputs.splitmix64(seed, k)
        c = [lib.gg_splitmix64(seed, int(x)) for x in k]
        assert [int(x) for x in py] == c


def test_uniform_range_and_moments():
    u = inputs.uniform(5, 200_000)
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 0.005 and abs(u.var() - 1 / 12) < 0.002
    assert np.array_equal(inputs.uniform(5, 10, offset=7), u[7:17])


def test_seed_samplers():
    off, col = inputs.rmat(14, seed=3)
    d = np.diff(off)
    s = inputs.seeds_deg2(off, 5000, 4)
    assert len(s) == 5000 and s.dtype == np.int32 and np.all(d[s] >= 2)
    assert np.array_equal(s, inputs.seeds_deg2(off, 5000, 4))
    x = inputs.config1_seed(off, col)
    nb = col[off[0]:off[1]]
    assert x in nb and d[x] == d[nb].max() and x == nb[d[nb] == d[nb].max()].min()
    e = inputs.eps_loguniform(20_000, 4, -8.0, -5.0)
    assert e.min() >= 1e-8 and e.max() < 1e-5
    assert abs(np.log10(e).mean() + 6.5) < 0.05
    t = inputs.poisson_arrivals(20_000, 100.0, 5)
    assert np.all(np.diff(t) > 0) and abs(t[-1] / len(t) - 0.01) < 0.0005
