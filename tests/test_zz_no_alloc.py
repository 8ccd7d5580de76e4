"""simrank_update_noalloc: the entry point for callers that cannot allocate
device memory when they apply an update (a host application whose device
memory belongs to another allocator, or a latency-bound loop that must not
stall on cudaMalloc/cudaFree).  Two updates in a row through it must give the
same S as the allocating path, simrank_apply_updates, and as the FP64 oracle
(Alg 1 per update), within the tolerances of the other GPU tests: 1e-6 with S
in FP32, 1e-10 with S in FP64; also at the size limits of its fixed scratch
array (n = 8192, K = 31).  Collected last on purpose."""
import ctypes

import numpy as np
import pytest

from oracle import simrank_oracle as O
from synth import chung_lu_digraph

pytestmark = pytest.mark.gpu

TOL32 = 1e-6
TOL64 = 1e-10


def in_csr(n, edges):
    rows = [[] for _ in range(n)]
    for a, b in edges:
        rows[b].append(a)
    rp = np.zeros(n + 1, np.int64)
    rp[1:] = np.cumsum([len(r) for r in rows])
    col = np.array([x for r in rows for x in r], np.int32)
    return rp, col


@pytest.fixture(scope="module")
def P():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__

    __graft_entry__.build()
    import paper_1711_00121_gb300 as P

    return P


def two_updates(n, s, d):
    edges = set(zip(s.tolist(), d.tolist()))
    deg = np.bincount(d, minlength=n)
    j1 = int(np.argmax(deg))
    i1 = next(x for x in range(n) if x != j1 and (x, j1) not in edges)
    i2, j2 = next((a, b) for a, b in sorted(edges) if deg[b] > 1 and b != j1)
    return edges, [(i1, j1, 1), (i2, j2, -1)]


def run_noalloc(P, n, S_host, prec, edges, ups, C, K):
    """Copies S to the device (n_pad x n_pad, zero padding), applies ups one
    call at a time through the C ABI and returns the device S."""
    import torch

    n_pad = (n + 127) // 128 * 128
    dt = torch.float32 if prec == 32 else torch.float64
    S = torch.zeros((n_pad, n_pad), dtype=dt, device="cuda")
    S[:n, :n] = torch.from_numpy(np.ascontiguousarray(S_host)).to(dt).cuda()
    stream = torch.cuda.current_stream()
    L = P.lib()
    cur = set(edges)
    for i, j, op in ups:
        new = cur | {(i, j)} if op > 0 else cur - {(i, j)}
        orp, ocol = in_csr(n, cur)
        nrp, ncol = in_csr(n, new)
        d_j = int(orp[j + 1] - orp[j])
        t = [torch.from_numpy(x).cuda() for x in (orp, ocol, nrp, ncol)]
        st = L.simrank_update_noalloc(n, n_pad, ctypes.c_void_p(S.data_ptr()), prec,
                                      *[ctypes.c_void_p(x.data_ptr()) for x in t],
                                      i, j, op, d_j, C, K, ctypes.c_void_p(stream.cuda_stream))
        assert st == 0, L.simrank_last_error(None)
        torch.cuda.synchronize()
        cur = new
    return S, t


def test_noalloc_two_updates_match_apply_updates(P):
    n, m, C, K = 1000, 8000, 0.6, 15
    s, d = chung_lu_digraph(n, m, 2.1, 2.1, 41)
    edges, ups = two_updates(n, s, d)
    ref = P.SimRank(n, s, d, C=C, K=K, s_precision=32, relabel=0)
    S0 = ref.dense(fp64=False)
    S, t = run_noalloc(P, n, S0, 32, edges, ups, C, K)
    ref.apply_updates(ups[:1])
    ref.apply_updates(ups[1:])
    want = ref.dense(fp64=False)
    got = S[:n, :n].cpu().numpy()
    assert float(np.max(np.abs(got.astype(np.float64) - want))) < TOL32
    # sizes above the fixed scratch array are rejected with a clear error
    L = P.lib()
    st = L.simrank_update_noalloc(9000, 9088, ctypes.c_void_p(S.data_ptr()), 32,
                                  *[ctypes.c_void_p(x.data_ptr()) for x in t],
                                  ups[0][0], ups[0][1], 1, 1, C, K, None)
    assert st == 1 and b"n must be" in L.simrank_last_error(None)
    st = L.simrank_update_noalloc(n, 1024, ctypes.c_void_p(S.data_ptr()), 32,
                                  *[ctypes.c_void_p(x.data_ptr()) for x in t],
                                  ups[0][0], ups[0][1], 1, 1, C, 32, None)
    assert st == 1 and b"K must be" in L.simrank_last_error(None)


@pytest.mark.parametrize("prec", [32, 64])
def test_noalloc_two_updates_match_oracle(P, prec):
    """Against Alg 1 in FP64 from the converged old S (the oracle, not the library)."""
    n, m, C, K = 900, 6000, 0.6, 12
    s, d = chung_lu_digraph(n, m, 2.1, 2.1, 42)
    edges, ups = two_updates(n, s, d)
    S0 = O.simrank_fixed_point(O.transition_matrix(n, s, d, sparse=True), C, tol=1e-15)
    S, _ = run_noalloc(P, n, S0, prec, edges, ups, C, K)
    want, _ = O.sequential_unit_updates(n, s, d, S0, ups, C, K)
    got = S[:n, :n].double().cpu().numpy()
    assert float(np.max(np.abs(got - want))) < (TOL32 if prec == 32 else TOL64)


def test_noalloc_at_its_limits_fp64(P):
    """n = 8192 and K = 31, the largest sizes of the fixed scratch array, with S
    in FP64 (old S from the library's FP64 initialisation, converged to 1e-13),
    on sampled columns against Alg 1 per update (oracle, column form) from the
    converged fixed point (Procedure 1 at K = 90)."""
    n, C, K = 8192, 0.6, 31
    s, d = chung_lu_digraph(n, 4 * n, 2.1, 2.1, 43)
    edges, ups = two_updates(n, s, d)
    h = P.SimRank(n, s, d, C=C, K=K, s_precision=64, relabel=0)
    S0 = h.dense()
    h.close()
    S, _ = run_noalloc(P, n, S0, 64, edges, ups, C, K)
    del S0
    rng = np.random.default_rng(44)
    query = sorted(set(rng.choice(n, 10, replace=False).tolist()) | {u[1] for u in ups})
    got = S[:n, query].cpu().numpy()
    Q0 = O.transition_matrix(n, s, d, sparse=True)
    want = O.alg1_stream_columns(n, s, d, lambda c: O.partial_sim_block(Q0, c, 90, C), ups, C, K,
                                 query)
    assert float(np.max(np.abs(got - want))) < TOL64
