"""simrank_update_noalloc: the entry point for callers that cannot allocate
device memory when they apply an update (a host application whose device
memory belongs to another allocator, or a latency-bound loop that must not
stall on cudaMalloc/cudaFree).  Two updates in a row through it must give the
same S as the allocating path, simrank_apply_updates, within the FP32
tolerance of the other GPU tests.  Collected last on purpose."""
import ctypes

import numpy as np
import pytest

from synth import chung_lu_digraph

pytestmark = pytest.mark.gpu

TOL32 = 1e-6


def in_csr(n, edges):
    rows = [[] for _ in range(n)]
    for a, b in edges:
        rows[b].append(a)
    rp = np.zeros(n + 1, np.int64)
    rp[1:] = np.cumsum([len(r) for r in rows])
    col = np.array([x for r in rows for x in r], np.int32)
    return rp, col


def test_noalloc_two_updates_match_apply_updates():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__

    __graft_entry__.build()
    import paper_1711_00121_gb300 as P

    n, m, C, K = 1000, 8000, 0.6, 15
    s, d = chung_lu_digraph(n, m, 2.1, 2.1, 41)
    edges = set(zip(s.tolist(), d.tolist()))
    deg = np.bincount(d, minlength=n)
    j1 = int(np.argmax(deg))
    i1 = next(x for x in range(n) if x != j1 and (x, j1) not in edges)
    i2, j2 = next((a, b) for a, b in sorted(edges) if deg[b] > 1 and b != j1)
    ups = [(i1, j1, 1), (i2, j2, -1)]

    ref = P.SimRank(n, s, d, C=C, K=K, s_precision=32, relabel=0)
    S0 = ref.dense(fp64=False)
    n_pad = (n + 127) // 128 * 128
    S = torch.zeros((n_pad, n_pad), dtype=torch.float32, device="cuda")
    S[:n, :n] = torch.from_numpy(np.ascontiguousarray(S0)).cuda()
    stream = torch.cuda.current_stream()
    L = P.lib()
    cur = set(edges)
    for i, j, op in ups:
        new = cur | {(i, j)} if op > 0 else cur - {(i, j)}
        orp, ocol = in_csr(n, cur)
        nrp, ncol = in_csr(n, new)
        d_j = int(orp[j + 1] - orp[j])
        t = [torch.from_numpy(x).cuda() for x in (orp, ocol, nrp, ncol)]
        st = L.simrank_update_noalloc(n, n_pad, ctypes.c_void_p(S.data_ptr()), 32,
                                      *[ctypes.c_void_p(x.data_ptr()) for x in t],
                                      i, j, op, d_j, C, K, ctypes.c_void_p(stream.cuda_stream))
        assert st == 0, L.simrank_last_error(None)
        torch.cuda.synchronize()
        cur = new
    ref.apply_updates(ups[:1])
    ref.apply_updates(ups[1:])
    want = ref.dense(fp64=False)
    got = S[:n, :n].cpu().numpy()
    assert float(np.max(np.abs(got.astype(np.float64) - want))) < TOL32
    # sizes above the fixed scratch array are rejected with a clear error
    st = L.simrank_update_noalloc(9000, 9088, ctypes.c_void_p(S.data_ptr()), 32,
                                  *[ctypes.c_void_p(x.data_ptr()) for x in t],
                                  i1, j1, 1, 1, C, K, None)
    assert st == 1 and b"n must be" in L.simrank_last_error(None)
