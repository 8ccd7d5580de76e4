"""The multi-GPU form of bench.py is N independent replicas (the update stream
is sequential; no data-path collective).  Its host logic runs here on CPU
with world size 2 over gloo: the timings reduce to their maximum over ranks on
every rank, and only rank 0 of the reference arm does work."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import sys

    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    # rank r timed 10 + r ms and 50 - r ms (e2e)
    out = bench.max_over_ranks([10.0 + rank, 50.0 - rank], dist)
    dist.barrier()
    q.put((rank, out))
    dist.destroy_process_group()


def test_max_over_ranks_world2_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    got = dict(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert got[0] == got[1] == [11.0, 50.0]


def test_max_over_ranks_single_process_is_identity():
    import sys

    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks([3.5, 7.25]) == [3.5, 7.25]


def test_reference_arm_other_ranks_do_nothing(capsys):
    import sys

    sys.path.insert(0, ROOT)
    import bench

    assert bench.run_reference(None, 1) is None
    assert capsys.readouterr().out == ""
