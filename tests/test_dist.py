"""Multi-process host logic on CPU (gloo, world size 2): the row partition
of a sharded GEMM and the one exchange step, the gather of fault reports
and counters."""
import os
import socket

import pytest

from paper_2305_01024_gb300 import dist as fd


@pytest.mark.parametrize("M,world,align", [(1000, 2, 128), (16384, 8, 128), (100, 4, 128), (777, 3, 120), (0, 2, 128)])
def test_partition_covers_rows_once_on_tile_boundaries(M, world, align):
    spans = [fd.partition_rows(M, world, r, align) for r in range(world)]
    covered = []
    for row0, rows in spans:
        assert rows >= 0
        if rows:
            assert row0 % align == 0
            covered += list(range(row0, row0 + rows))
    assert covered == list(range(M))
    sizes = [-(-rows // align) for _, rows in spans]
    assert max(sizes) - min(sizes) <= 1  # balanced to within one tile


def test_partition_rejects_bad_arguments():
    with pytest.raises(ValueError):
        fd.partition_rows(10, 0, 0)
    with pytest.raises(ValueError):
        fd.partition_rows(10, 2, 2)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        M = 1000
        row0, rows = fd.partition_rows(M, world, rank, 128)
        recs = [{"tile_m": 0, "tile_n": 1, "row": 5 + rank, "col": 7, "kind": 0, "delta": 2.0 ** 10},
                {"tile_m": 0, "tile_n": 0, "row": -1, "col": 3, "kind": 2, "delta": 1.0}]
        merged = fd.gather_records(recs, row0)
        counts = fd.sum_counts({"detected": 2, "corrected": 1 + rank, "false_alarms": 0})
        q.put((rank, row0, rows, merged, counts))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_gather_reports_and_counts():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = {}
    for _ in procs:
        rank, row0, rows, merged, counts = q.get(timeout=120)
        out[rank] = (row0, rows, merged, counts)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0a, na, ma, ca), (r0b, nb, mb, cb) = out[0], out[1]
    assert (r0a, na) == (0, 512) and (r0b, nb) == (512, 488)
    assert ma == mb  # every rank gets the same merged report
    located = [(r["rank"], r["row"], r["col"]) for r in ma if r["kind"] == 0]
    assert located == [(0, 5, 7), (1, 512 + 6, 7)]  # rows in global coordinates
    assert sum(1 for r in ma if r["row"] == -1) == 2  # no row: not shifted
    assert ca == cb == {"corrected": 3, "detected": 4, "false_alarms": 0}
