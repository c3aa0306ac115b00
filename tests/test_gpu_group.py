"""The persistent tensor-core kernel over a table of problems, against the
CPU oracle: single GEMMs with more tiles than SMs (both TMEM accumulators and
their phases in use), groups of ragged bf16 / e4m3 problems, faults located
per problem, and a CUDA graph that captures the grouped call and replays it.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu
U32 = 2.0 ** -24
TDM, TDN = 125, 252  # bf16 data tile of C when checksums ride in the MMA tile (ftgemm_tc_tile)


@pytest.fixture(scope="module")
def ft():
    import torch
    import paper_2305_01024_gb300 as ft
    assert torch.cuda.is_available()
    ft.lib()
    return ft


@pytest.fixture(params=[False, True], ids=["cta", "pair"])
def handle(ft, request):
    # every test runs on single CTAs and on CTA pairs (cta_group::2 MMAs),
    # which must give the same tiles, checksums and records
    h = ft.Handle(0)
    h.set_tc_pair(request.param)
    yield h
    h.close()


def _sched(orc, K):
    return orc.Schedule(m_tb=TDM, n_tb=TDN, k_tb=64, m_w=TDM, n_w=TDN, m_t=TDM, n_t=TDN,
                        cadence=-(-K // 64), split_k=1, level=orc.TILE, lam=32.0, u=U32)


def _int_problem(M, N, K, seed):
    A = synth.integers((M, K), seed).astype(np.float32)
    B = synth.integers((K, N), seed + 1).astype(np.float32)
    Cin = synth.integers((M, N), seed + 2).astype(np.float32)
    return A, B, Cin


def _dev_bf16(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda().to(torch.bfloat16)


@pytest.mark.parametrize("level", ["off", "tile"])
def test_persistent_many_tiles_per_cta_exact(ft, handle, orc, level):
    """4096 x 2048 x 192: 35 x 9 = 315 tiles at level TILE (16 x 8 = 128 at
    OFF, then 4096 x 4096), so CTAs run two or three tiles and reuse both
    accumulators; integer inputs make every sum exact."""
    import torch
    M, N, K = (4096, 2048, 192) if level == "tile" else (4096, 4096, 192)
    A, B, Cin = _int_problem(M, N, K, 4100)
    dC = torch.from_numpy(Cin.copy()).cuda()
    rep = handle.gemm(_dev_bf16(A), _dev_bf16(B), dC, alpha=1.0, beta=-2.0, level=ft.LEVELS[level],
                      dtype=ft.BF16)
    torch.cuda.synchronize()
    ref = orc.gemm_ref(A, B, 1.0, -2.0, Cin)
    assert np.array_equal(dC.cpu().numpy().astype(np.float64), ref)
    assert rep.detected == 0


def test_persistent_faults_in_late_tiles_match_oracle(ft, handle, orc):
    """Faults in tiles that CTAs reach second or third (list entries >= the
    CTA count) are located and corrected exactly as the oracle does."""
    import torch
    M, N, K = 4096, 2048, 192
    A, B, _ = _int_problem(M, N, K, 4200)
    tiles_m, tiles_n = -(-M // TDM), -(-N // TDN)
    nks = -(-K // 64)
    pos = synth.fault_positions(synth.workload_seed("group512", 30), 12, tiles_m, tiles_n, nks, TDM, TDN, M, N, nks)
    faults = [(tm, tn, ks, r, c, float(2 ** 10)) for (tm, tn, ks, r, c) in pos]
    dC = torch.zeros(M, N, device="cuda")
    rep = handle.gemm(_dev_bf16(A), _dev_bf16(B), dC, level=ft.FT_TILE, dtype=ft.BF16, inject=faults)
    torch.cuda.synchronize()
    res = orc.gemm_ft(A, B, _sched(orc, K), faults=faults)
    assert np.array_equal(dC.cpu().numpy().astype(np.float64), res.C)
    got = sorted((r["tile_m"], r["tile_n"], r["row"], r["col"], r["kind"], r["delta"]) for r in rep.records)
    want = sorted((o.tile_m, o.tile_n, o.row, o.col, o.kind, o.delta) for o in res.records)
    assert got == want and rep.corrected == len(faults)


def _ragged_shapes(n, seed):
    u = synth.unit(seed, 3 * n).reshape(n, 3)
    shapes = []
    for a, b, c in u:
        shapes.append((1 + int(a * 700), 1 + int(b * 700), 8 * (1 + int(c * 80))))
    shapes[0] = (1, 1, 8)          # degenerate: one element
    shapes[1] = (TDM, TDN, 64)     # exactly one tile
    shapes[2] = (TDM + 1, TDN + 1, 72)  # one tile plus a ragged row and column
    return shapes


def _make_group(ft, handle, shapes, seed, level, faults=None):
    import torch
    host, dev = [], []
    for q, (M, N, K) in enumerate(shapes):
        A, B, Cin = _int_problem(M, N, K, seed + 10 * q)
        alpha, beta = (1.0, 0.0) if q % 2 == 0 else (2.0, -1.0)
        dA, dB = _dev_bf16(A), _dev_bf16(B)
        dC = torch.from_numpy(Cin.copy()).cuda()
        host.append((A, B, Cin, alpha, beta))
        dev.append((dA, dB, dC, alpha, beta))
    grp = ft.Group(handle, dev, dtype=ft.BF16, level=ft.LEVELS[level])
    if faults:
        grp.set_faults(faults)
    return grp, host, dev


@pytest.mark.parametrize("level", ["off", "tile"])
def test_group_ragged_bf16_exact(ft, handle, orc, level):
    import torch
    shapes = _ragged_shapes(24, 5100)
    grp, host, dev = _make_group(ft, handle, shapes, 5200, level)
    tm, tn = grp.tiles()
    dm, dn = (TDM, TDN) if level == "tile" else (128, 256)
    assert tm == [-(-M // dm) for (M, N, K) in shapes] and tn == [-(-N // dn) for (M, N, K) in shapes]
    grp.run()
    torch.cuda.synchronize()
    for (A, B, Cin, alpha, beta), (_, _, dC, _, _) in zip(host, dev):
        ref = orc.gemm_ref(A, B, alpha, beta, Cin)
        assert np.array_equal(dC.cpu().numpy().astype(np.float64), ref)
    assert handle.report_fetch().detected == 0
    grp.close()


def test_group_faults_per_problem_match_oracle(ft, handle, orc):
    import torch
    shapes = _ragged_shapes(16, 5300)
    faults, per_problem = [], {}
    for q, (M, N, K) in enumerate(shapes):
        if q % 3 != 1:
            continue
        tiles_m, tiles_n, nks = -(-M // TDM), -(-N // TDN), -(-K // 64)
        # at most one fault per tile: the tile is the unit, verified once
        nf = min(2, tiles_m * tiles_n)
        for (a, b, ks, r, c) in synth.fault_positions(synth.workload_seed("group512", 40 + q), nf, tiles_m, tiles_n, nks,
                                                      TDM, TDN, M, N, nks):
            faults.append((q, a, b, ks, r, c, 2.0 ** 9))
            per_problem.setdefault(q, []).append((a, b, ks, r, c, 2.0 ** 9))
    grp, host, dev = _make_group(ft, handle, shapes, 5400, "tile", faults)
    grp.run()
    torch.cuda.synchronize()
    rep = handle.report_fetch()
    got = sorted((r["problem"], r["tile_m"], r["tile_n"], r["row"], r["col"], r["kind"]) for r in rep.records)
    want = []
    for q, ((A, B, Cin, alpha, beta), (_, _, dC, _, _)) in enumerate(zip(host, dev)):
        res = orc.gemm_ft(A, B, _sched(orc, A.shape[1]), faults=per_problem.get(q, ()), alpha=alpha,
                          beta=beta, Cin=Cin)
        assert np.array_equal(dC.cpu().numpy().astype(np.float64), res.C)
        want += [(q, o.tile_m, o.tile_n, o.row, o.col, o.kind) for o in res.records]
    assert got == sorted(want) and rep.corrected == len(faults)
    grp.close()


def test_group_fp8_within_bound(ft, handle, orc):
    import torch
    shapes = [(300, 500, 256), (64, 1000, 512), (777, 129, 384)]
    dev, host = [], []
    for q, (M, N, K) in enumerate(shapes):
        A = synth.normal((M, K), synth.workload_seed("group512", 50 + q))
        B = synth.normal((K, N), synth.workload_seed("group512", 60 + q))
        dA, sa = handle.quantize(torch.from_numpy(A).cuda(), ft.E4M3)
        dB, sb = handle.quantize(torch.from_numpy(np.ascontiguousarray(B)).cuda(), ft.E4M3)
        _, Aq, _ = orc.quant_e4m3(A)
        _, Bq, _ = orc.quant_e4m3(B)
        dC = torch.zeros(M, N, device="cuda")
        dev.append((dA, dB, dC, 1.0, 0.0, sa, sb))
        host.append((Aq, Bq, sa, sb))
    grp = ft.Group(handle, dev, dtype=ft.E4M3, level=ft.FT_TILE)
    grp.run()
    torch.cuda.synchronize()
    for (Aq, Bq, sa, sb), d in zip(host, dev):
        K = Aq.shape[1]
        s = np.float64(np.float32(sa)) * np.float64(np.float32(sb))
        ref = orc.gemm_ref(Aq, Bq) * s
        absprod = np.abs(Aq) @ np.abs(Bq)
        bound = 2 * K * U32 * absprod * s + 4 * U32 * np.abs(ref)
        assert np.all(np.abs(d[2].cpu().numpy().astype(np.float64) - ref) <= bound)
    assert handle.report_fetch().detected == 0
    grp.close()


def test_group_captured_in_cuda_graph_replays(ft, orc):
    """The grouped call enqueues without host synchronisation, so a CUDA graph
    captures it; each replay recomputes every C and adds its fault events to
    the handle's report."""
    import torch
    stream = torch.cuda.Stream()
    h = ft.Handle(0, stream=stream)
    shapes = _ragged_shapes(10, 5500)
    M0, N0, K0 = shapes[3]
    faults = [(3, 0, 0, 0, min(5, M0 - 1), min(7, N0 - 1), 2.0 ** 8)]
    grp, host, dev = _make_group(ft, h, shapes, 5600, "tile", faults)
    torch.cuda.synchronize()
    # beta is nonzero for odd problems: reset C to its input before each replay
    c_in = [torch.from_numpy(Cin.copy()).cuda() for (_, _, Cin, _, _) in host]
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=stream):
        grp.run()
    for rep_i in range(2):
        for (_, _, dC, _, _), ci in zip(dev, c_in):
            dC.copy_(ci)
        torch.cuda.synchronize()
        graph.replay()
        torch.cuda.synchronize()
        for (A, B, Cin, alpha, beta), (_, _, dC, _, _) in zip(host, dev):
            ref = orc.gemm_ref(A, B, alpha, beta, Cin)
            assert np.array_equal(dC.cpu().numpy().astype(np.float64), ref)
    rep = h.report_fetch()
    assert rep.corrected == 2 and all(r["problem"] == 3 for r in rep.records)
    grp.close()
    h.close()
