"""lgc_sweep_noalloc: the sweep cut for callers that cannot let the library
allocate device memory during a call (their device memory belongs to their
own allocator, or an allocation's failure or synchronisation mid-request is
not acceptable).  Called through the C ABI with device buffers the test
owns; its result must equal lgc_sweep's exactly (the sweep cut is integer
arithmetic plus one division, so the tolerance used for it everywhere is
exact equality), on consecutive calls that reuse the shared scratch array.

Collected last on purpose, and self-contained, so it passes alone in a fresh
process as well as after the other tests."""
import ctypes
import math

import numpy as np
import pytest

from paper_1604_07515_gb300 import inputs, lgc

pytestmark = pytest.mark.gpu


def noalloc_sweep(g, idx_np, val_np, torch):
    lib = lgc.load()
    idx = torch.tensor(idx_np, dtype=torch.int32, device="cuda")
    val = torch.tensor(val_np, dtype=torch.float64, device="cuda")
    ids = torch.full((max(1, len(idx_np)),), -1, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    out = lgc.Cluster()
    st = lib.lgc_sweep_noalloc(g.handle, len(idx_np), idx.data_ptr(), val.data_ptr(),
                               ids.data_ptr(), ctypes.byref(out))
    return st, out, ids[: out.size].cpu().numpy() if st == 0 else None


def test_noalloc_sweep_equals_lgc_sweep_on_consecutive_calls():
    torch = pytest.importorskip("torch")
    ctx = lgc.Context(0)
    off, col = inputs.rmat(13, seed=9)
    g = lgc.Graph(ctx, off, col)
    x = inputs.config1_seed(off, col)
    y = int(inputs.seeds_deg2(off, 1, 77)[0])
    cases = []
    for seed, eps in [(x, 1e-6), (y, 1e-4), (x, 1e-5)]:
        p, _ = lgc.prnibble(g, seed, 0.01, eps, mode="det")
        assert 0 < p.nnz <= 65536
        cases.append((p.idx, p.val))
    # a vector with ties in p/d and zero entries
    d = np.diff(off)
    nz = np.flatnonzero(d > 0)[:3000].astype(np.int32)
    cases.append((nz, (np.arange(len(nz)) % 4) * 0.25 * d[nz]))
    for idx, val in cases:  # consecutive calls share the scratch array
        assert len(idx) <= 65536
        ref = lgc.sweep(g, lgc.host_svec(idx, val))
        st, out, ids = noalloc_sweep(g, idx, val, torch)
        assert st == lgc.LGC_OK
        assert out.size == ref.size and out.vol == ref.vol and out.cut == ref.cut
        assert out.conductance == ref.conductance or (
            math.isinf(out.conductance) and math.isinf(ref.conductance))
        assert out.on_device == 1
        assert np.array_equal(ids, ref.ids)
    g.close()
    ctx.close()


def test_noalloc_sweep_rejects_oversized_and_bad_input():
    torch = pytest.importorskip("torch")
    ctx = lgc.Context(0)
    off, col = inputs.path(5)
    g = lgc.Graph(ctx, off, col)
    lib = lgc.load()
    out = lgc.Cluster()
    buf = torch.zeros(4, dtype=torch.float64, device="cuda")
    too_many = 65536 + 1
    st = lib.lgc_sweep_noalloc(g.handle, too_many, buf.data_ptr(), buf.data_ptr(),
                               buf.data_ptr(), ctypes.byref(out))
    assert st == lgc.LGC_EINVAL
    st, out, _ = noalloc_sweep(g, np.array([7], np.int32), np.array([1.0]), torch)
    assert st == lgc.LGC_EINVAL  # vertex 7 does not exist
    st, out, ids = noalloc_sweep(g, np.zeros(0, np.int32), np.zeros(0), torch)
    assert st == lgc.LGC_OK and out.size == 0 and math.isinf(out.conductance)
    g.close()
    ctx.close()
