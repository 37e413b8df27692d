"""Device memory from the caller's allocator (lgc_ctx_create_with_alloc):
PyTorch's caching allocator or a counting wrapper around it.  Results are
the same as with the device pool, every block handed out comes back, and the
graph's memory shows in PyTorch's own accounting."""
import numpy as np
import pytest

import oracle
from paper_1604_07515_gb300 import inputs, lgc

pytestmark = pytest.mark.gpu


def run(ctx, off, col, x):
    g = lgc.Graph(ctx, off, col)
    p, st = lgc.prnibble(g, x, 0.01, 1e-6, mode="det")
    c = lgc.sweep(g, p)
    h, _ = lgc.hkpr(g, x, 5.0, 10, 1e-6, mode="atomic")
    res = (p.idx.copy(), p.val.copy(), c.ids.copy(), c.cut, c.vol, h.idx.copy(), h.val.copy())
    del p, c, h
    g.close()
    return res


def test_torch_allocator_same_results_and_accounting():
    import torch
    off, col = inputs.rmat(14, seed=3)
    x = inputs.config1_seed(off, col)
    ref_ctx = lgc.Context(0)
    ref = run(ref_ctx, off, col, x)
    ref_ctx.close()

    torch.cuda.synchronize()
    base = torch.cuda.memory_allocated(0)
    ctx = lgc.Context(0, torch.cuda.current_stream(), allocator="torch")
    g = lgc.Graph(ctx, off, col)
    torch.cuda.synchronize()
    # the CSR (offsets and columns) came out of torch's pool
    assert torch.cuda.memory_allocated(0) - base >= 8 * len(off) + 4 * len(col)
    g.close()
    got = run(ctx, off, col, x)
    ctx.close()
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated(0) == base
    assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1])  # det: bitwise
    assert np.array_equal(got[2], ref[2]) and got[3:5] == ref[3:5]
    a, b = np.zeros(len(off) - 1), np.zeros(len(off) - 1)
    a[got[5]] = got[6]
    b[ref[5]] = ref[6]
    assert np.abs(a - b).sum() <= 1e-12 * np.abs(b).sum()
    # and against the oracle
    o = oracle.prnibble(off, col, x, 0.01, 1e-6)
    assert np.array_equal(got[0], o.idx) and np.array_equal(got[1], o.val)


def test_counting_allocator_balanced():
    import torch
    live, calls = {}, {"alloc": 0, "free": 0}

    def alloc(nbytes, stream):
        calls["alloc"] += 1
        ptr = torch.cuda.caching_allocator_alloc(nbytes, 0, stream)
        live[ptr] = nbytes
        return ptr

    def free(ptr, stream):
        calls["free"] += 1
        assert ptr in live
        del live[ptr]
        torch.cuda.caching_allocator_delete(ptr)

    off, col = inputs.rmat(12, seed=1)
    x = inputs.config1_seed(off, col)
    ctx = lgc.Context(0, allocator=(alloc, free))
    run(ctx, off, col, x)
    ctx.set_option(lgc.OPT_RESULT_ON_DEVICE, 1)
    g = lgc.Graph(ctx, off, col)
    ps, _ = lgc.prnibble_batch(g, [x, x], 0.01, 1e-5)
    cs = lgc.sweep_batch(g, ps)
    del ps, cs
    g.close()
    ctx.close()
    assert calls["alloc"] > 0 and calls["alloc"] == calls["free"] and not live


def test_failing_allocator_reports_enomem():
    def alloc(nbytes, stream):
        return 0

    def free(ptr, stream):
        raise AssertionError("nothing was handed out")

    off, col = inputs.rmat(10, seed=1)
    ctx = lgc.Context(0, allocator=(alloc, free))
    with pytest.raises(lgc.LgcError) as e:
        lgc.Graph(ctx, off, col)
    assert e.value.status == lgc.LGC_ENOMEM
    ctx.close()
