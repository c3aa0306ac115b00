"""Multi-GPU host logic: one process per GPU, no collective on the data path.

Output tiles of C are independent (the checksums of a tile involve only the
rows of A and the columns of B it uses, Eq. 1-3), so a GEMM shards over
ranks by blocks of C rows with no exchange during the computation.  The one
exchange is the fault report: every rank's records are gathered so that the
whole job's detections can be counted and located in global coordinates.

The functions take a torch.distributed process group (NCCL on GPUs, gloo in
the CPU tests) and move only small host objects.
"""
from __future__ import annotations


def partition_rows(M: int, world: int, rank: int, align: int = 128):
    """Rows [row0, row0 + rows) of an M-row GEMM for `rank` of `world`:
    contiguous blocks of whole `align`-row tiles (the ragged last tile goes to
    the last non-empty rank), as even as the tiles allow."""
    if world <= 0 or not 0 <= rank < world or M < 0 or align <= 0:
        raise ValueError("bad partition arguments")
    tiles = -(-M // align)
    base, extra = divmod(tiles, world)
    t0 = rank * base + min(rank, extra)
    nt = base + (1 if rank < extra else 0)
    row0 = min(M, t0 * align)
    rows = max(0, min(M, (t0 + nt) * align) - row0)
    return row0, rows


def gather_records(records, row0: int = 0, group=None):
    """All ranks' fault records (dicts as returned by Handle.report_fetch),
    rows shifted by each rank's `row0`, each tagged with its rank; every rank
    gets the same merged list, sorted by (row, col, rank, kind)."""
    import torch.distributed as dist
    mine = []
    for r in records:
        g = dict(r)
        if g.get("row", -1) >= 0:
            g["row"] = g["row"] + row0
        mine.append(g)
    if dist.is_available() and dist.is_initialized():
        world = dist.get_world_size(group)
        rank = dist.get_rank(group)
        everyone = [None] * world
        dist.all_gather_object(everyone, (rank, mine), group=group)
    else:
        everyone = [(0, mine)]
    merged = []
    for rank, recs in everyone:
        for r in recs:
            g = dict(r)
            g["rank"] = rank
            merged.append(g)
    merged.sort(key=lambda r: (r.get("row", -1), r.get("col", -1), r["rank"], r.get("kind", 0)))
    return merged


def sum_counts(counts: dict, group=None) -> dict:
    """Element-wise sum of integer counters over all ranks (same keys on
    every rank)."""
    import torch
    import torch.distributed as dist
    keys = sorted(counts)
    if not (dist.is_available() and dist.is_initialized()):
        return {k: int(counts[k]) for k in keys}
    backend = dist.get_backend(group)
    device = "cuda" if backend == "nccl" else "cpu"
    t = torch.tensor([int(counts[k]) for k in keys], dtype=torch.int64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return {k: int(v) for k, v in zip(keys, t.tolist())}
