"""A group rebound to a DEVICE array of problems (ftgemm_grouped_gemm_dev):
the operands are read from device memory when the call runs, so a captured
graph follows whatever the array holds at replay time.

Integer-valued operands (exact in bf16 and e4m3, every sum exact in fp32)
make every C comparable bit for bit with the oracle's plain product.  Checked:
the rebound operands are the ones computed (and the creation ones are left
alone), faults set on the group are located in the rebound problems, a graph
replays with the array's new contents, an entry that breaks a rebinding rule
is skipped (its C untouched, the report's fetch returns FTGEMM_ERR_ARG) until
a valid rebinding, and B read in place by the MMA (bf16, level OFF) is
re-pointed too.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

TDM, TDN = {"bf16": 125, "e4m3": 123}, {"bf16": 252, "e4m3": 248}  # data tile with checksums (ftgemm_tc_tile)
# K a multiple of 16 (A's rows 16-byte aligned for TMA in bf16 and e4m3); N
# mixes bf16 rows that are and are not 16-byte multiples (B read in place or
# through B^T at level OFF)
SHAPES = [(300, 500, 256), (128, 130, 80), (1000, 260, 640), (64, 64, 64), (250, 1200, 144), (777, 333, 1008)]


@pytest.fixture(scope="module")
def ft():
    import torch
    import paper_2305_01024_gb300 as ft
    assert torch.cuda.is_available()
    ft.lib()
    return ft


def _operands(seed, dtype_name, scales=(1.0, 1.0)):
    """Host integer operands and the device problems of the group's shapes:
    A, B on {-4..4}, C_in on {-4..4} (C = A B - C_in)."""
    import torch
    host, dev = [], []
    for q, (M, N, K) in enumerate(SHAPES):
        A = synth.integers((M, K), seed + 3 * q).astype(np.float32)
        B = synth.integers((K, N), seed + 3 * q + 1).astype(np.float32)
        Cin = synth.integers((M, N), seed + 3 * q + 2).astype(np.float32)
        tA, tB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
        if dtype_name == "bf16":
            tA, tB = tA.to(torch.bfloat16), tB.to(torch.bfloat16)
        else:  # e4m3 codes of the integers (exact)
            tA = tA.to(torch.float8_e4m3fn).view(torch.uint8)
            tB = tB.to(torch.float8_e4m3fn).view(torch.uint8)
        host.append((A, B, Cin))
        dev.append((tA, tB, torch.from_numpy(Cin.copy()).cuda(), 1.0, -1.0, scales[0], scales[1]))
    return host, dev


def _expect(orc, host, scales=(1.0, 1.0)):
    s = scales[0] * scales[1]
    return [orc.gemm_ref(A, B, alpha=s, beta=-1.0, Cin=Cin) for A, B, Cin in host]


def _check_all(dev, want, skip=()):
    for q, (pr, w) in enumerate(zip(dev, want)):
        got = pr[2].cpu().numpy().astype(np.float64)
        if q in skip:
            continue
        assert np.array_equal(got, w), f"problem {q}"


@pytest.mark.parametrize("dtype_name,level_name", [("bf16", "FT_TILE"), ("bf16", "FT_OFF"), ("e4m3", "FT_TILE")])
def test_rebound_operands_are_the_ones_computed(ft, orc, dtype_name, level_name):
    import torch
    dtype = ft.BF16 if dtype_name == "bf16" else ft.E4M3
    level = getattr(ft, level_name)
    h = ft.Handle(0)
    hx, dx = _operands(synth.workload_seed("group512", 300), dtype_name)
    # the rebound set has other values and, for e4m3, other scales
    sy = (1.0, 1.0) if dtype_name == "bf16" else (2.0, 1.0)
    hy, dy = _operands(synth.workload_seed("group512", 400), dtype_name, sy)
    g = ft.Group(h, dx, dtype=dtype, level=level)
    faults = []
    if level == ft.FT_TILE:
        # offsets far above the threshold, set on the group (they follow the binding)
        faults = [(0, 0, 0, -1, 5, 7, 1024.0), (2, 1, 0, -1, 30, 100, -2048.0), (5, 5, 1, -1, 50, 0, 512.0)]
        g.set_faults(faults)
    table = ft.problem_table(dy)
    g.run_device(table)
    rep = h.report_fetch()
    _check_all(dy, _expect(orc, hy, sy))
    # the creation operands were not touched
    for (A, B, Cin), pr in zip(hx, dx):
        assert np.array_equal(pr[2].cpu().numpy(), Cin)
    if faults:
        got = sorted((r["problem"], r["row"], r["col"], r["kind"]) for r in rep.records)
        want = sorted((f[0], f[1] * TDM[dtype_name] + f[4], f[2] * TDN[dtype_name] + f[5], 0) for f in faults)
        assert got == want and rep.corrected == len(faults)
    else:
        assert rep.detected == 0
    # a plain call afterwards computes on the operands last bound
    for pr in dy:
        pr[2].copy_(torch.zeros_like(pr[2]))
    g.run()
    h.report_fetch()
    wz = [orc.gemm_ref(A, B, alpha=sy[0] * sy[1], beta=-1.0, Cin=np.zeros_like(Cin)) for A, B, Cin in hy]
    _check_all(dy, wz)
    g.close()
    h.close()


def test_graph_replays_follow_the_array(ft, orc):
    import torch
    h = ft.Handle(0)
    hx, dx = _operands(synth.workload_seed("group512", 310), "bf16")
    hy, dy = _operands(synth.workload_seed("group512", 410), "bf16")
    hz, dz = _operands(synth.workload_seed("group512", 510), "bf16")
    g = ft.Group(h, dx, dtype=ft.BF16, level=ft.FT_TILE)
    table = ft.problem_table(dy)
    table_z = ft.problem_table(dz)
    side = torch.cuda.Stream()
    main = torch.cuda.current_stream()
    graph = torch.cuda.CUDAGraph()
    h.set_stream(side)
    with torch.cuda.graph(graph, stream=side):
        g.run_device(table)
    h.set_stream(main)
    graph.replay()
    torch.cuda.synchronize()
    h.report_fetch()
    _check_all(dy, _expect(orc, hy))
    # new contents of the same array: the next replay computes the new problems
    y_after = [pr[2].clone() for pr in dy]
    table.copy_(table_z)
    graph.replay()
    torch.cuda.synchronize()
    h.report_fetch()
    _check_all(dz, _expect(orc, hz))
    for a, pr in zip(y_after, dy):
        assert torch.equal(a, pr[2])
    del graph
    g.close()
    h.close()


def test_entry_breaking_a_rule_is_skipped(ft, orc):
    import torch
    h = ft.Handle(0)
    hx, dx = _operands(synth.workload_seed("group512", 320), "bf16")
    hy, dy = _operands(synth.workload_seed("group512", 420), "bf16")
    g = ft.Group(h, dx, dtype=ft.BF16, level=ft.FT_TILE)
    bad = ft.problem_structs(dy)
    bad[2].m += 1  # sizes differ from the group's: rule 1
    table = torch.frombuffer(bytearray(bytes(bad)), dtype=torch.int64).cuda()
    sentinel = torch.full_like(dy[2][2], 7.0)
    dy[2][2].copy_(sentinel)
    g.run_device(table)
    with pytest.raises(ft.FtgemmError) as ei:
        h.report_fetch()
    assert ei.value.status == ft.ERR_ARG
    want = _expect(orc, hy)
    _check_all(dy, want, skip=(2,))
    assert torch.equal(dy[2][2], sentinel)
    # the problem stays skipped for plain calls until a valid rebinding
    g.run()
    h.report_fetch()
    assert torch.equal(dy[2][2], sentinel)
    for q in range(len(dy)):
        dy[q][2].copy_(torch.from_numpy(hy[q][2]).cuda())
    g.run_device(ft.problem_table(dy))
    rep = h.report_fetch()
    assert rep.detected == 0
    _check_all(dy, want)
    g.close()
    h.close()
