"""lgc_sweep_noalloc: the sweep cut for callers that cannot let the library
allocate device memory during a call -- their device memory belongs to their
own allocator (a serving process that reserved the GPU's memory up front),
or an allocation's out-of-memory failure or device synchronisation in the
middle of a request is not acceptable.

Called through the C ABI with device buffers the test owns.  Its result must
equal lgc_sweep's and the oracle's exactly (the sweep cut is integer
arithmetic plus one division, so exact equality is the tolerance used for it
everywhere), on consecutive calls that reuse the shared scratch array, up to
the documented limit of LGC_SWEEP_NOALLOC_MAX_N entries; a repeated vertex
is rejected as lgc_sweep rejects it; and the device's free memory does not
move across calls.

Collected last on purpose, and self-contained, so it passes alone in a fresh
process as well as after the other tests."""
import ctypes
import math

import numpy as np
import pytest

import oracle
from paper_1604_07515_gb300 import inputs, lgc

pytestmark = pytest.mark.gpu

MAX_N = 65536  # LGC_SWEEP_NOALLOC_MAX_N in include/lgc.h


class DeviceCase:
    """Device buffers of one input vector and its output, allocated up front
    so that the calls themselves run with nothing else allocating."""

    def __init__(self, torch, idx_np, val_np):
        self.idx_np, self.val_np = idx_np, val_np
        self.idx = torch.tensor(idx_np, dtype=torch.int32, device="cuda")
        self.val = torch.tensor(val_np, dtype=torch.float64, device="cuda")
        self.ids = torch.full((max(1, len(idx_np)),), -1, dtype=torch.int32, device="cuda")

    def call(self, g):
        out = lgc.Cluster()
        st = lgc.load().lgc_sweep_noalloc(g.handle, len(self.idx_np), self.idx.data_ptr(),
                                          self.val.data_ptr(), self.ids.data_ptr(),
                                          ctypes.byref(out))
        return st, out

    def ids_host(self, out):
        return self.ids[: out.size].cpu().numpy()


def same_cluster(out, ids, size, vol, cut, phi, ref_ids):
    assert out.size == size and out.vol == vol and out.cut == cut
    assert out.conductance == phi or (math.isinf(out.conductance) and math.isinf(phi))
    assert out.on_device == 1
    assert np.array_equal(ids, ref_ids)


def test_noalloc_sweep_equals_lgc_sweep_and_oracle_on_consecutive_calls():
    torch = pytest.importorskip("torch")
    ctx = lgc.Context(0)
    off, col = inputs.rmat(17, seed=9)
    g = lgc.Graph(ctx, off, col)
    x = inputs.config1_seed(off, col)
    y = int(inputs.seeds_deg2(off, 1, 77)[0])
    vecs = []
    for seed, eps in [(x, 1e-6), (y, 1e-4), (x, 1e-5)]:
        p, _ = lgc.prnibble(g, seed, 0.01, eps, mode="det")
        assert 0 < p.nnz <= MAX_N
        vecs.append((p.idx.copy(), p.val.copy()))
    d = np.diff(off)
    nz = np.flatnonzero(d > 0).astype(np.int32)
    # a short vector with ties in p/d and zero entries (the one-block sort)
    vecs.append((nz[:700], (np.arange(700) % 4) * 0.25 * d[nz[:700]]))
    # exactly the limit: 65536 entries over vertices of many degrees, keys
    # p/d in {0, 1/4, 1/2, 3/4} (zeros leave the support, the rest tie in
    # threes of thousands and are ordered by id), so the sort spans all 32
    # of its tiles and the scans their longest runs
    big = nz[:MAX_N]
    assert len(big) == MAX_N
    vecs.append((big, (np.arange(MAX_N) % 4) * 0.25 * d[big]))
    # a full-length vector with distinct keys
    vecs.append((big, (1.0 + np.arange(MAX_N)[::-1]) * d[big] / MAX_N))
    cases = [DeviceCase(torch, i, v) for i, v in vecs]
    refs = []
    for c in cases:
        rs = oracle.sweep(off, col, c.idx_np, c.val_np)
        cl = lgc.sweep(g, lgc.host_svec(c.idx_np, c.val_np))
        assert (cl.size, cl.vol, cl.cut) == (rs.best, rs.best_vol, rs.best_cut)
        assert np.array_equal(cl.ids, rs.cluster) and cl.conductance == rs.conductance
        refs.append(rs)
    torch.cuda.synchronize()

    def run_all():
        for c, rs in zip(cases, refs):
            st, out = c.call(g)
            assert st == lgc.LGC_OK
            same_cluster(out, c.ids_host(out), rs.best, rs.best_vol, rs.best_cut,
                         rs.conductance, rs.cluster)

    run_all()  # first calls: the driver loads this code and reserves the array
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(2):  # two more calls in a row per vector, on the shared array
        run_all()
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0, "device memory moved during a call"
    g.close()
    ctx.close()


def test_noalloc_sweep_rejects_oversized_repeated_and_bad_input():
    torch = pytest.importorskip("torch")
    ctx = lgc.Context(0)
    off, col = inputs.path(5)
    g = lgc.Graph(ctx, off, col)
    lib = lgc.load()
    out = lgc.Cluster()
    buf = torch.zeros(4, dtype=torch.float64, device="cuda")
    st = lib.lgc_sweep_noalloc(g.handle, MAX_N + 1, buf.data_ptr(), buf.data_ptr(),
                               buf.data_ptr(), ctypes.byref(out))
    assert st == lgc.LGC_EINVAL
    st, out = DeviceCase(torch, np.array([7], np.int32), np.array([1.0])).call(g)
    assert st == lgc.LGC_EINVAL  # vertex 7 does not exist
    # a vertex named twice: rejected, as lgc_sweep rejects it
    rep_idx, rep_val = np.array([1, 1], np.int32), np.array([0.5, 0.25])
    with pytest.raises(lgc.LgcError) as e:
        lgc.sweep(g, lgc.host_svec(rep_idx, rep_val))
    assert e.value.status == lgc.LGC_EINVAL
    st, out = DeviceCase(torch, rep_idx, rep_val).call(g)
    assert st == lgc.LGC_EINVAL
    st, out = DeviceCase(torch, np.array([0, 2, 2, 3], np.int32),
                         np.array([0.1, 0.2, 0.3, 0.4])).call(g)
    assert st == lgc.LGC_EINVAL
    # the next valid call is unaffected by the rejected ones
    c = DeviceCase(torch, np.array([1, 2], np.int32), np.array([0.5, 0.25]))
    st, out = c.call(g)
    rs = oracle.sweep(off, col, c.idx_np, c.val_np)
    assert st == lgc.LGC_OK
    same_cluster(out, c.ids_host(out), rs.best, rs.best_vol, rs.best_cut, rs.conductance,
                 rs.cluster)
    st, out = DeviceCase(torch, np.zeros(0, np.int32), np.zeros(0)).call(g)
    assert st == lgc.LGC_OK and out.size == 0 and math.isinf(out.conductance)
    g.close()
    ctx.close()
