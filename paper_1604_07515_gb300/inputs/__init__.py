"""Seeded synthetic inputs: graphs, seeds and parameters.

This module holds no clustering arithmetic.  Both the CUDA library's tests
and the CPU oracle take their inputs from here, so neither side produces the
other's inputs.

Graphs are undirected CSR pairs ``(off: int64[n+1], col: int32[2m])`` with
sorted adjacency lists, no self loops and no duplicate edges, matching the
paper's inputs (Sec. 4, "Input Graphs").

* ``rmat(scale, ...)``      R-MAT power-law graphs standing in for the
  paper's social and web graphs (soc-LJ, Orkut, Twitter, friendster, Yahoo),
  which are not available here.
* ``paper_example()``       the 8-vertex, 8-edge graph of Fig. fig:conductance,
  completed from the Z array printed in Sec. 3.1's sweep example.
* ``path``, ``star``, ``clique_pair``, ``grid3d``: small hand-built graphs.
* ``config1_seed``, ``seeds_deg2``, ``eps_loguniform``, ``poisson_arrivals``:
  seed and parameter samplers (counter-based SplitMix64).
"""
from __future__ import annotations

import ctypes
import functools
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "graphgen.c")
_LIB = os.path.join(_HERE, "libgraphgen.so")
_lock = threading.Lock()
_lib = None

RMAT_A, RMAT_B, RMAT_C = 0.57, 0.19, 0.19


def build(force: bool = False) -> str:
    with _lock:
        if (not force and os.path.exists(_LIB)
                and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
            return _LIB
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-O2", "-fPIC", "-shared", "-pthread", "-o", tmp, _SRC],
                       check=True)
        os.replace(tmp, _LIB)
        return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        lib.gg_rmat.restype = ctypes.c_void_p
        lib.gg_rmat.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                ctypes.c_double, ctypes.c_uint64, ctypes.c_int]
        lib.gg_n.restype = ctypes.c_int64
        lib.gg_n.argtypes = [ctypes.c_void_p]
        lib.gg_nnz.restype = ctypes.c_int64
        lib.gg_nnz.argtypes = [ctypes.c_void_p]
        lib.gg_copy.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
        lib.gg_free.argtypes = [ctypes.c_void_p]
        lib.gg_splitmix64.restype = ctypes.c_uint64
        lib.gg_splitmix64.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
        _lib = lib
    return _lib


@functools.lru_cache(maxsize=4)
def rmat(scale: int, edge_factor: int = 16, seed: int = 1, a: float = RMAT_A,
         b: float = RMAT_B, c: float = RMAT_C, threads: int | None = None):
    """Symmetrised R-MAT graph (no self loops, no duplicates, sorted CSR)."""
    lib = _load()
    nt = threads or min(16, os.cpu_count() or 1)
    h = lib.gg_rmat(scale, edge_factor, a, b, c, seed, nt)
    if not h:
        raise MemoryError(f"R-MAT scale {scale} generation failed")
    n, nnz = lib.gg_n(h), lib.gg_nnz(h)
    off = np.empty(n + 1, dtype=np.int64)
    col = np.empty(nnz, dtype=np.int32)
    lib.gg_copy(h, off.ctypes.data, col.ctypes.data)
    lib.gg_free(h)
    off.setflags(write=False)
    col.setflags(write=False)
    return off, col


def splitmix64(seed: int, k: np.ndarray) -> np.ndarray:
    """Word k of the counter-based SplitMix64 stream `seed` (vectorised)."""
    k = np.asarray(k, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + (k + np.uint64(1)) * np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


def uniform(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """`count` doubles in [0, 1) with 53 random bits each."""
    w = splitmix64(seed, np.arange(offset, offset + count, dtype=np.uint64))
    return (w >> np.uint64(11)).astype(np.float64) * 2.0 ** -53


def from_edges(n: int, edges) -> tuple[np.ndarray, np.ndarray]:
    """Undirected CSR from an edge list (symmetrised, deduplicated, sorted)."""
    e = np.asarray(edges, dtype=np.int64).reshape(-1, 2)
    e = e[e[:, 0] != e[:, 1]]
    both = np.concatenate([e, e[:, ::-1]], axis=0)
    keys = np.unique(both[:, 0] * n + both[:, 1]) if len(both) else np.zeros(0, np.int64)
    src, dst = keys // n, keys % n
    off = np.zeros(n + 1, dtype=np.int64)
    np.add.at(off, src + 1, 1)
    off = np.cumsum(off).astype(np.int64)
    return off, dst.astype(np.int32)


def paper_example():
    """Fig. fig:conductance graph, n = 8, m = 8, as A..H = 0..7.

    The figure itself is not available; its edges among A..D and D's three
    outside neighbours are read off the Z array of Sec. 3.1's worked example
    (A: B, C; B: A, C; C: A, B, D; D: C and three vertices outside
    {A, B, C, D}).  The eighth edge (G-H) joins two outside vertices; any such
    choice leaves the example's degrees, volumes and cuts unchanged.
    """
    A, B, C, D, E, F, G, H = range(8)
    return from_edges(8, [(A, B), (A, C), (B, C), (C, D), (D, E), (D, F), (D, G), (G, H)])


def path(n: int):
    return from_edges(n, [(i, i + 1) for i in range(n - 1)])


def star(leaves: int):
    return from_edges(leaves + 1, [(0, i) for i in range(1, leaves + 1)])


def clique_pair(k: int):
    """Two k-cliques joined by one edge (0 -- k)."""
    e = [(i, j) for i in range(k) for j in range(i + 1, k)]
    e += [(k + i, k + j) for i in range(k) for j in range(i + 1, k)]
    e.append((0, k))
    return from_edges(2 * k, e)


def grid3d(side: int):
    """3-D torus: every vertex joined to its two neighbours in each dimension
    (the paper's 3D-grid input, Sec. 4)."""
    n = side ** 3
    idx = np.arange(n).reshape(side, side, side)
    e = []
    for ax in range(3):
        e.append(np.stack([idx.ravel(), np.roll(idx, -1, axis=ax).ravel()], axis=1))
    return from_edges(n, np.concatenate(e))


def random_graph(n: int, m: int, seed: int):
    """Erdos-Renyi-style multigraph sample (deduplicated), for small tests."""
    u = uniform(seed, 2 * m)
    e = np.stack([(u[:m] * n).astype(np.int64), (u[m:] * n).astype(np.int64)], axis=1)
    return from_edges(n, e)


def degrees(off) -> np.ndarray:
    return np.diff(np.asarray(off))


def config1_seed(off, col) -> int:
    """Vertex 0's highest-degree neighbour (ties: lowest id)."""
    nb = np.asarray(col[off[0]:off[1]])
    d = degrees(off)[nb]
    return int(nb[np.flatnonzero(d == d.max())].min())


def seeds_deg2(off, count: int, seed: int) -> np.ndarray:
    """`count` vertices drawn uniformly (with replacement) among those of degree >= 2."""
    cand = np.flatnonzero(degrees(off) >= 2)
    u = uniform(seed, count)
    return cand[np.minimum((u * len(cand)).astype(np.int64), len(cand) - 1)].astype(np.int32)


def eps_loguniform(count: int, seed: int, lo_exp: float = -8.0, hi_exp: float = -5.0,
                   offset: int = 0) -> np.ndarray:
    """eps = 10^(lo + (hi - lo) u)."""
    return 10.0 ** (lo_exp + (hi_exp - lo_exp) * uniform(seed, count, offset))


def poisson_arrivals(count: int, rate: float, seed: int) -> np.ndarray:
    """Arrival times (s) of an open-loop Poisson process: gaps -ln(1-u)/rate."""
    gaps = -np.log1p(-uniform(seed, count)) / rate
    return np.cumsum(gaps)
