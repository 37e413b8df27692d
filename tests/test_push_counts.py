"""Sequential versus synchronous PR-Nibble push counts (the analogue of the
paper's table of pushes and iterations, Sec. 3.3), computed by the oracle on
R-MAT graphs and a 3-D torus at alpha = 0.01, eps = 1e-7.  The synchronous
rounds may push more than the sequential queue; both stay within the
work bound sum of pushed degrees <= 1/(alpha eps), and both end with every
residual below eps d(v)."""
import numpy as np
import pytest

import oracle
from paper_1604_07515_gb300 import inputs

ALPHA, EPS = 0.01, 1e-7


@pytest.mark.parametrize("name", ["rmat14", "grid20"])
def test_sequential_vs_synchronous_pushes(name):
    off, col = inputs.rmat(14, seed=1) if name == "rmat14" else inputs.grid3d(20)
    x = inputs.config1_seed(off, col)
    seq = oracle.prnibble_queue(off, col, x, ALPHA, EPS)
    syn = oracle.prnibble(off, col, x, ALPHA, EPS)
    d = np.diff(off)
    for r in (seq, syn):
        assert r.pushed_edges <= 1.0 / (ALPHA * EPS)  # Sec. 3.3 work bound
        assert r.pushes > 0
    # both leave every residual below the threshold (idx2/val2: r)
    for r in (seq, syn):
        if len(r.idx2):
            assert np.all(r.val2 < EPS * d[r.idx2])
    ratio = syn.pushes / seq.pushes
    print(f"{name}: sequential {seq.pushes} pushes, synchronous {syn.pushes} pushes "
          f"in {syn.rounds} rounds, ratio {ratio:.3f}")
    assert 0.5 < ratio < 3.0
