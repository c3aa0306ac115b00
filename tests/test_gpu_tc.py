"""Parity of the tensor-core (tcgen05 / TMEM) path with the CPU oracle:
bf16 and fp8 E4M3 operands, fp32 accumulation, the plain GEMM and the
tile-level ABFT whose checksums ride through the MMA; the operand quantizer
against the oracle's RNE / OCP E4M3 rounding."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu
U32 = 2.0 ** -24


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


# With checksums on, the last 3 (bf16) or 5 (e4m3) rows and as many columns
# of the 128 x 256 MMA tile carry the checksum pieces (the data columns a
# multiple of 4): a CTA computes a 125 x 252 (bf16) or 123 x 248 (e4m3) tile
# of C.
TDM, TDN = {"bf16": 125, "fp8": 123}, {"bf16": 252, "fp8": 248}


def _tc_sched(orc, K, dt):
    bk = 64 if dt == "bf16" else 128
    nks = -(-K // bk)
    dm, dn = TDM[dt], TDN[dt]
    return orc.Schedule(m_tb=dm, n_tb=dn, k_tb=bk, m_w=dm, n_w=dn, m_t=dm, n_t=dn,
                        cadence=nks, split_k=1, level=orc.TILE, lam=32.0, u=U32)


def _bf16_inputs(orc, kind, M, N, K, seed):
    A = synth.make(kind, (M, K), seed)
    B = synth.make(kind, (K, N), seed + 1)
    return orc.round_bf16(A).astype(np.float32), orc.round_bf16(B).astype(np.float32)


def _run_bf16(ft, handle, A, B, Cin, alpha, beta, level):
    import torch
    dA = torch.from_numpy(A).cuda().to(torch.bfloat16)
    dB = torch.from_numpy(B).cuda().to(torch.bfloat16)
    dC = torch.from_numpy(Cin.copy()).cuda()
    rep = handle.gemm(dA, dB, dC, alpha=alpha, beta=beta, level=level, dtype=ft.BF16)
    torch.cuda.synchronize()
    return dC.cpu().numpy().astype(np.float64), rep


def _bound(A, B, Cin, alpha, beta, K):
    absprod = np.abs(A.astype(np.float64)) @ np.abs(B.astype(np.float64))
    return 2 * K * U32 * (abs(alpha) * absprod + abs(beta) * np.abs(Cin.astype(np.float64)))


@pytest.mark.parametrize("level", ["off", "tile"])
# N a multiple of 8: B is read in place (MN-major), including ragged last tiles (264, 504);
# N = 300, 260: B goes through the transposed copy
@pytest.mark.parametrize("shape", [(256, 512, 320), (200, 300, 136), (128, 256, 64), (130, 260, 72),
                                   (200, 264, 136), (136, 504, 200), (125, 252, 64), (126, 253, 72),
                                   (376, 760, 128), (250, 504, 64)])
def test_tc_bf16_integers_exact(ft, handle, orc, level, shape):
    M, N, K = shape
    A, B = _bf16_inputs(orc, "int", M, N, K, 500 + M)
    Cin = synth.integers((M, N), 600 + N)
    lv = ft.LEVELS[level]
    C, rep = _run_bf16(ft, handle, A, B, Cin, 2.0, -1.0, lv)
    ref = 2 * (A.astype(np.int64) @ B.astype(np.int64)) - Cin.astype(np.int64)
    assert np.array_equal(C, ref)
    assert rep.detected == 0
    if lv == ft.FT_TILE:
        res = orc.gemm_ft(A, B, _tc_sched(orc, K, "bf16"), alpha=2.0, beta=-1.0, Cin=Cin)
        assert np.array_equal(res.C, ref) and res.detected == 0


@pytest.mark.parametrize("shape,lda", [((130, 264, 75), 80), ((300, 500, 331), 336), ((64, 100, 13), 16)])
def test_tc_bf16_ragged_k_strided_a_exact(ft, handle, orc, shape, lda):
    """K not a multiple of 8, A a row-strided view into a wider buffer: the
    encode pass's last 8-element group of each row straddles K (elements
    past K, which lie inside A's padded rows, must not count), and N
    multiples of 4 but not of 8 put a B group across N as well."""
    import torch
    M, N, K = shape
    A, B = _bf16_inputs(orc, "int", M, N, K, 900 + K)
    Cin = synth.integers((M, N), 901 + K)
    buf = torch.full((M, lda), 3.0, dtype=torch.bfloat16, device="cuda")  # nonzero padding
    buf[:, :K] = torch.from_numpy(A).cuda().to(torch.bfloat16)
    dA = buf[:, :K]
    dB = torch.from_numpy(B).cuda().to(torch.bfloat16)
    ref = A.astype(np.int64) @ B.astype(np.int64) + Cin.astype(np.int64)
    for lv in (ft.FT_OFF, ft.FT_TILE):
        dC = torch.from_numpy(Cin.copy()).cuda()
        rep = handle.gemm(dA, dB, dC, alpha=1.0, beta=1.0, level=lv, dtype=ft.BF16)
        torch.cuda.synchronize()
        assert np.array_equal(dC.cpu().numpy().astype(np.float64), ref)
        assert rep.detected == 0


@pytest.mark.parametrize("level", ["off", "tile"])
def test_tc_bf16_normal_within_bound(ft, handle, orc, level):
    M, N, K = 384, 512, 1024
    A, B = _bf16_inputs(orc, "normal", M, N, K, synth.workload_seed("tc_square", 0))
    Cin = synth.normal((M, N), synth.workload_seed("tc_square", 2))
    C, rep = _run_bf16(ft, handle, A, B, Cin, 1.0, 0.5, ft.LEVELS[level])
    ref = orc.gemm_ref(A, B, 1.0, 0.5, Cin)
    assert np.all(np.abs(C - ref) <= _bound(A, B, Cin, 1.0, 0.5, K))
    assert rep.detected == 0


def test_quantize_matches_oracle(ft, handle, orc):
    import torch
    x = synth.normal((4096 + 7,), 77) * 3.0
    dx = torch.from_numpy(x).cuda()
    yb, sb = handle.quantize(dx, ft.BF16)
    assert sb == 1.0
    assert np.array_equal(yb.float().cpu().numpy().astype(np.float64), orc.round_bf16(x))
    y8, s8 = handle.quantize(dx, ft.E4M3)
    deq, q, scale = orc.quant_e4m3(x)
    assert np.float32(s8) == np.float32(scale)
    codes = y8.cpu().numpy()
    got = torch.from_numpy(codes).view(torch.float8_e4m3fn).to(torch.float64).numpy()
    assert np.array_equal(got, q)


@pytest.mark.parametrize("level", ["off", "tile"])
def test_tc_fp8_normal_within_bound(ft, handle, orc, level):
    import torch
    M, N, K = 256, 512, 1024
    A = synth.normal((M, K), synth.workload_seed("tc_square", 10))
    B = synth.normal((K, N), synth.workload_seed("tc_square", 11))
    dA8, sa = handle.quantize(torch.from_numpy(A).cuda(), ft.E4M3)
    # B is quantized as the K x N matrix it is
    dB8, sb = handle.quantize(torch.from_numpy(np.ascontiguousarray(B)).cuda(), ft.E4M3)
    _, Aq, _ = orc.quant_e4m3(A)
    _, Bq, _ = orc.quant_e4m3(B)
    handle.set_fp8_scales(sa, sb)
    dC = torch.zeros(M, N, device="cuda")
    rep = handle.gemm(dA8, dB8, dC, alpha=1.0, beta=0.0, level=ft.LEVELS[level], dtype=ft.E4M3)
    torch.cuda.synchronize()
    C = dC.cpu().numpy().astype(np.float64)
    ref = orc.gemm_ref(Aq, Bq) * (np.float64(np.float32(sa)) * np.float64(np.float32(sb)))
    bound = _bound(Aq, Bq, np.zeros((M, N)), 1.0, 0.0, K) * (sa * sb) + 4 * U32 * np.abs(ref)
    assert np.all(np.abs(C - ref) <= bound)
    assert rep.detected == 0


@pytest.mark.parametrize("shape", [(246, 496, 256), (250, 500, 320), (123, 248, 128), (7, 9, 128), (130, 760, 128)])
def test_tc_e4m3_integers_exact(ft, handle, orc, shape):
    """E4M3 codes of integers in [-4, 4] (exact in the format) with unit
    scales: C, the checksums and every partial sum are exact in fp32, so C
    equals the int64 product bit for bit at both levels, and at TILE the
    records of seeded faults of +-2^10 (one per tile, 123 x 248 tiles) equal
    the oracle's, with C restored exactly."""
    import torch
    M, N, K = shape
    A = synth.integers((M, K), 710 + M)
    B = synth.integers((K, N), 720 + N)
    dA = torch.from_numpy(A).cuda().to(torch.float8_e4m3fn)
    dB = torch.from_numpy(np.ascontiguousarray(B)).cuda().to(torch.float8_e4m3fn)
    handle.set_fp8_scales(1.0, 1.0)
    ref = A.astype(np.int64) @ B.astype(np.int64)
    for level in ("off", "tile"):
        dC = torch.zeros(M, N, device="cuda")
        rep = handle.gemm(dA, dB, dC, alpha=1.0, beta=0.0, level=ft.LEVELS[level], dtype=ft.E4M3)
        torch.cuda.synchronize()
        assert np.array_equal(dC.cpu().numpy().astype(np.int64), ref) and rep.detected == 0
    sched = _tc_sched(orc, K, "fp8")
    tm_n, tn_n, nks = -(-M // TDM["fp8"]), -(-N // TDN["fp8"]), -(-K // 128)
    pos = synth.fault_positions(synth.workload_seed("tc_square", 50), tm_n * tn_n, tm_n, tn_n, nks,
                                TDM["fp8"], TDN["fp8"], M, N, nks)
    faults = [(tm, tn, ks, r, c, 1024.0 if (tm + tn) % 2 == 0 else -1024.0) for (tm, tn, ks, r, c) in pos]
    dC = torch.zeros(M, N, device="cuda")
    rep = handle.gemm(dA, dB, dC, alpha=1.0, beta=0.0, level=ft.FT_TILE, dtype=ft.E4M3, inject=faults)
    torch.cuda.synchronize()
    res = orc.gemm_ft(A, B, sched, faults=faults)
    assert np.array_equal(dC.cpu().numpy().astype(np.int64), ref) and np.array_equal(res.C, ref)
    key = lambda r: (r["tile_m"], r["tile_n"], r["row"], r["col"], r["kind"], r["delta"]) if isinstance(r, dict) \
        else (r.tile_m, r.tile_n, r.row, r.col, r.kind, r.delta)
    assert sorted(map(key, rep.records)) == sorted(map(key, res.records))
    assert rep.corrected == len(faults) == res.corrected


@pytest.mark.parametrize("dt", ["bf16", "fp8"])
def test_tc_faults_located_and_corrected(ft, handle, orc, dt):
    """Seeded faults in several tiles (the tensor-core square workload's, reduced): every fault is
    flagged at its element, corrected, and C matches the fault-free result
    within the bound; the records match the oracle's (tile-level unit, one
    verification after the last k-step)."""
    import torch
    M, N, K = 384, 768, 1024
    A = synth.normal((M, K), synth.workload_seed("tc_square", 20))
    B = synth.normal((K, N), synth.workload_seed("tc_square", 21))
    if dt == "bf16":
        Aq = orc.round_bf16(A).astype(np.float32)
        Bq = orc.round_bf16(B).astype(np.float32)
        dA = torch.from_numpy(Aq).cuda().to(torch.bfloat16)
        dB = torch.from_numpy(Bq).cuda().to(torch.bfloat16)
        dtype, sc = ft.BF16, 1.0
    else:
        dA, sa = handle.quantize(torch.from_numpy(A).cuda(), ft.E4M3)
        dB, sb = handle.quantize(torch.from_numpy(B).cuda(), ft.E4M3)
        _, Aq, _ = orc.quant_e4m3(A)
        _, Bq, _ = orc.quant_e4m3(B)
        handle.set_fp8_scales(1.0, 1.0)
        dtype, sc = ft.E4M3, 1.0
    sched = _tc_sched(orc, K, dt)
    ksteps = -(-K // sched.k_tb)
    AB = Aq.astype(np.float64) @ Bq.astype(np.float64)
    pos = synth.fault_positions(synth.workload_seed("tc_square", 22), 5, 3, 3, ksteps, TDM[dt], TDN[dt], M, N, ksteps)
    mags = synth.log_uniform(synth.workload_seed("tc_square", 23), 5, 1e-2, 1e3)
    faults = []
    for (tm, tn, ks, r, c), g in zip(pos, mags):
        tmax = np.abs(AB[tm * TDM[dt]:(tm + 1) * TDM[dt], tn * TDN[dt]:(tn + 1) * TDN[dt]]).max()
        faults.append((tm, tn, ks, r, c, float(np.float32(g * tmax))))
    dC = torch.zeros(M, N, device="cuda")
    rep = handle.gemm(dA, dB, dC, level=ft.FT_TILE, dtype=dtype, inject=faults)
    torch.cuda.synchronize()
    C = dC.cpu().numpy().astype(np.float64)
    res = orc.gemm_ft(Aq, Bq, sched, faults=faults)
    key = lambda r: (r["tile_m"], r["tile_n"], r["row"], r["col"], r["kind"]) if isinstance(r, dict) \
        else (r.tile_m, r.tile_n, r.row, r.col, r.kind)
    assert sorted(map(key, rep.records)) == sorted(map(key, res.records))
    assert rep.corrected == len(faults) == res.corrected
    for o in res.records:
        assert abs(o.delta) > 4 * o.tau
    slack = np.zeros_like(C)
    for o in res.records:
        slack[o.row, o.col] = o.tau
    assert np.all(np.abs(C - res.C) <= _bound(Aq, Bq, np.zeros_like(C), 1.0, 0.0, K) + slack)


def test_tc_checksum_hit_and_seu_violation(ft, handle, orc):
    import torch
    M, N, K = 128, 256, 512
    A = synth.integers((M, K), 31)
    B = synth.integers((K, N), 32)
    dA = torch.from_numpy(A).cuda().to(torch.bfloat16)
    dB = torch.from_numpy(B).cuda().to(torch.bfloat16)
    sched = _tc_sched(orc, K, "bf16")
    for faults, kind in [([(0, 0, 2, 10, 20, 64.0, 1)], 2), ([(0, 0, 2, 10, 200, 64.0, 2)], 2),
                         ([(0, 0, 1, 3, 4, 64.0), (0, 0, 5, 70, 90, 32.0)], 1)]:
        dC = torch.zeros(M, N, device="cuda")
        rep = handle.gemm(dA, dB, dC, level=ft.FT_TILE, dtype=ft.BF16, inject=faults)
        torch.cuda.synchronize()
        res = orc.gemm_ft(A, B, sched, faults=faults)
        assert np.array_equal(dC.cpu().numpy().astype(np.float64), res.C)
        assert [(r["row"], r["col"], r["kind"]) for r in rep.records] == \
            [(r.row, r.col, r.kind) for r in res.records]
        assert rep.records[0]["kind"] == kind
        assert rep.records[0]["delta"] == res.records[0].delta
