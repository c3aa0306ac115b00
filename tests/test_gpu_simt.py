"""Parity of the fp32 SIMT fused-ABFT SGEMM (through the C ABI) with the CPU
oracle: bit-exact C and fault records on integer-valued inputs, stated
tolerances on floating-point inputs, every level and every compiled tile
tuple, ragged tiles, the scalar (unaligned) path, split-K, checksum hits,
violations of the single-event-upset model and argument errors."""
import zlib

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

TUPLES = {
    "wide": (128, 128, 16, 64, 64, 16, 8),
    "wide32": (128, 128, 32, 64, 64, 16, 8),
    "huge16": (128, 128, 16, 32, 64, 8, 8),
    "huge": (128, 128, 8, 32, 64, 8, 8),
    "large": (64, 64, 8, 32, 64, 8, 8),
    "tall": (32, 128, 8, 16, 64, 4, 8),
    "medium": (32, 32, 8, 16, 32, 4, 4),
    "small": (16, 16, 16, 8, 16, 2, 2),
}
LEVELS = {"thread": 1, "warp": 2, "block": 3}
U32 = 2.0 ** -24


@pytest.fixture(scope="module")
def ft():
    import torch
    import paper_2305_01024_gb300 as ft
    assert torch.cuda.is_available()
    ft.lib()  # raises if the CUDA library is missing
    return ft


@pytest.fixture()
def handle(ft):
    h = ft.Handle(0)
    yield h
    h.close()


def _sched(name, cadence=4, split_k=1):
    m_tb, n_tb, k_tb, m_w, n_w, m_t, n_t = TUPLES[name]
    return dict(m_tb=m_tb, n_tb=n_tb, k_tb=k_tb, m_w=m_w, n_w=n_w, m_t=m_t, n_t=n_t,
                cadence=cadence, split_k=split_k)


def _oracle_sched(orc, s, level, lam=32.0):
    return orc.Schedule(m_tb=s["m_tb"], n_tb=s["n_tb"], k_tb=s["k_tb"], m_w=s["m_w"], n_w=s["n_w"],
                        m_t=s["m_t"], n_t=s["n_t"], cadence=s["cadence"], split_k=s["split_k"],
                        level=level, lam=lam, u=U32)


def _unit_fn(s, level):
    m_w, n_w, m_t, n_t = s["m_w"], s["n_w"], s["m_t"], s["n_t"]
    if level == 3:
        return lambda r, c: 0
    if level == 2:
        return lambda r, c: (r // m_w, c // n_w)
    lm, ln = m_w // m_t, n_w // n_t
    vm, vn = min(4, m_t), min(4, n_t)
    return lambda r, c: (r // m_w, (r % m_w) % (lm * vm) // vm, c // n_w, (c % n_w) % (ln * vn) // vn)


def _run(ft, handle, A, B, Cin, alpha, beta, level, s, faults):
    import torch
    handle.set_schedule(s)
    dA = torch.from_numpy(A).cuda()
    dB = torch.from_numpy(B).cuda()
    dC = torch.from_numpy(Cin.copy()).cuda()
    rep = handle.gemm(dA, dB, dC, alpha=alpha, beta=beta, level=level, inject=faults,
                      capacity=1 << 14)
    torch.cuda.synchronize()
    return dC.cpu().numpy().astype(np.float64), rep


def _key(r):
    if isinstance(r, dict):
        return (r["tile_m"], r["tile_n"], r["kstep"], r["row"], r["col"], r["kind"])
    return (r.tile_m, r.tile_n, r.kstep, r.row, r.col, r.kind)


def _compare_exact(rep, res):
    assert (rep.detected, rep.corrected, rep.uncorrectable, rep.checksum_only) == \
        (res.detected, res.corrected, res.uncorrectable, res.checksum_only)
    assert [_key(r) for r in rep.records] == [_key(r) for r in res.records]
    for g, o in zip(rep.records, res.records):
        assert g["delta"] == o.delta and g["residual_r"] == o.residual_r and g["residual_c"] == o.residual_c
        assert g["tau"] == pytest.approx(o.tau, rel=1e-4, abs=1e-30)


# ---------------------------------------------------------------------------
# integer-valued inputs: everything is exact, so GPU == oracle bit for bit
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("level", ["block", "warp", "thread"])
def test_int256_bit_exact(ft, handle, orc, level):
    """M=N=K=256, integers in [-4,4], 4 faults of +2^10 at seeded (tile, k-step, element)."""
    M = N = K = 256
    A = synth.integers((M, K), synth.workload_seed("int256", 0))
    B = synth.integers((K, N), synth.workload_seed("int256", 1))
    Cin = np.zeros((M, N), np.float32)
    lv = LEVELS[level]
    s = _sched("huge", cadence=4)
    pos = synth.fault_positions(synth.workload_seed("int256", 2), 4, 2, 2, 32, 128, 128, M, N, 4,
                                unit_of=_unit_fn(s, lv))
    faults = [p + (1024.0,) for p in pos]
    C, rep = _run(ft, handle, A, B, Cin, 1.0, 0.0, lv, s, faults)
    res = orc.gemm_ft(A, B, _oracle_sched(orc, s, lv), faults=faults)
    assert np.array_equal(C, res.C)
    assert np.array_equal(C, A.astype(np.int64) @ B.astype(np.int64))
    _compare_exact(rep, res)
    assert rep.corrected == 4


@pytest.mark.parametrize("tup", list(TUPLES))
@pytest.mark.parametrize("level", ["off", "thread", "warp", "block"])
@pytest.mark.parametrize("aligned", [True, False])
def test_tuples_levels_ragged_exact(ft, handle, orc, tup, level, aligned):
    """Every compiled tile tuple and level, several tiles with ragged tails,
    vector (aligned) and scalar (odd sizes) paths, alpha/beta, faults."""
    M, N, K = (200, 168, 136) if aligned else (203, 171, 133)
    seed = zlib.crc32(f"{tup}/{level}/{aligned}".encode()) % 10_000
    A = synth.integers((M, K), 1000 + seed)
    B = synth.integers((K, N), 2000 + seed)
    Cin = synth.integers((M, N), 3000 + seed)
    lv = {"off": 0, **LEVELS}[level]
    s = _sched(tup, cadence=3)
    mt, nt, kt = s["m_tb"], s["n_tb"], s["k_tb"]
    tiles_m, tiles_n, ksteps = -(-M // mt), -(-N // nt), -(-K // kt)
    faults = []
    if lv:
        pos = synth.fault_positions(4000 + seed, 6, tiles_m, tiles_n, ksteps, mt, nt, M, N, 3,
                                    unit_of=_unit_fn(s, lv))
        faults = [p + (float(2 ** (6 + q)),) for q, p in enumerate(pos)]
    C, rep = _run(ft, handle, A, B, Cin, -2.0, 3.0, lv, s, faults)
    ref = -2 * (A.astype(np.int64) @ B.astype(np.int64)) + 3 * Cin.astype(np.int64)
    assert np.array_equal(C, ref)
    if lv:
        res = orc.gemm_ft(A, B, _oracle_sched(orc, s, lv), faults=faults, alpha=-2.0, beta=3.0, Cin=Cin)
        assert np.array_equal(res.C, ref)
        _compare_exact(rep, res)
        assert rep.corrected == len(faults)
    else:
        assert rep.detected == 0


@pytest.mark.parametrize("level", ["thread", "warp", "block"])
@pytest.mark.parametrize("target", [1, 2])
def test_checksum_hit(ft, handle, orc, level, target):
    M = N = 128
    K = 64
    A = synth.integers((M, K), 71)
    B = synth.integers((K, N), 72)
    lv = LEVELS[level]
    s = _sched("huge", cadence=2)
    faults = [(0, 0, 3, 37, 90, 256.0, target)]
    C, rep = _run(ft, handle, A, B, np.zeros((M, N), np.float32), 1.0, 0.0, lv, s, faults)
    res = orc.gemm_ft(A, B, _oracle_sched(orc, s, lv), faults=faults)
    assert np.array_equal(C, A.astype(np.int64) @ B.astype(np.int64))
    _compare_exact(rep, res)
    assert rep.checksum_only == 1 and rep.detected == 1


@pytest.mark.parametrize("level", ["thread", "warp", "block"])
def test_seu_violation_is_uncorrectable(ft, handle, orc, level):
    M = N = K = 128
    A = synth.integers((M, K), 81)
    B = synth.integers((K, N), 82)
    lv = LEVELS[level]
    s = _sched("huge", cadence=4)
    # two faults in the same thread fragment (rows 0/16, cols 0/32 of thread (0,0))
    faults = [(0, 0, 1, 0, 0, 64.0), (0, 0, 2, 16, 32, 32.0)]
    C, rep = _run(ft, handle, A, B, np.zeros((M, N), np.float32), 1.0, 0.0, lv, s, faults)
    res = orc.gemm_ft(A, B, _oracle_sched(orc, s, lv), faults=faults)
    assert np.array_equal(C, res.C)
    _compare_exact(rep, res)
    assert rep.uncorrectable >= 1 and rep.corrected == 0


def test_split_k_exact(ft, handle, orc):
    """Long K with split-K: each split verifies its own partial."""
    M = N = 128
    K = 8192
    A = synth.integers((M, K), 91)
    B = synth.integers((K, N), 92)
    s = _sched("huge", cadence=32, split_k=8)
    faults = [(0, 0, 5, 1, 2, 512.0), (0, 0, 700, 100, 3, -512.0), (0, 0, -1, 127, 127, 1024.0)]
    C, rep = _run(ft, handle, A, B, np.zeros((M, N), np.float32), 1.0, 0.0, 3, s, faults)
    res = orc.gemm_ft(A, B, _oracle_sched(orc, s, 3), faults=faults)
    assert np.array_equal(C, A.astype(np.int64) @ B.astype(np.int64))
    _compare_exact(rep, res)
    assert rep.corrected == 3


@pytest.mark.parametrize("split", [3, 5, 6])
def test_split_k_not_a_power_of_two(ft, handle, orc, split):
    """Split counts the autotuner may pick to fill the SMs' CTA slots, on a
    ragged K: every split verifies its own partial, faults near split edges."""
    M, N = 200, 130
    K = 16 * 301 + 7  # 302 k-steps of 16, the last one short
    A = synth.integers((M, K), 95 + split)
    B = synth.integers((K, N), 96 + split)
    s = _sched("wide", cadence=8, split_k=split)
    per = -(-302 // split)
    faults = [(0, 0, per - 1, 3, 4, 256.0), (1, 1, per, 70, 1, -512.0), (0, 1, 301, 127, 1, 1024.0)]
    C, rep = _run(ft, handle, A, B, np.zeros((M, N), np.float32), 1.0, 0.0, 3, s, faults)
    res = orc.gemm_ft(A, B, _oracle_sched(orc, s, 3), faults=faults)
    assert np.array_equal(C, A.astype(np.int64) @ B.astype(np.int64))
    _compare_exact(rep, res)
    assert rep.corrected == 3


def test_degenerate_shapes(ft, handle, orc):
    for (M, N, K) in [(1, 1, 1), (1, 5, 3), (7, 1, 2), (3, 3, 17)]:
        A = synth.integers((M, K), 100 + M)
        B = synth.integers((K, N), 200 + N)
        for name in ("huge", "small"):
            s = _sched(name, cadence=1)
            C, rep = _run(ft, handle, A, B, np.zeros((M, N), np.float32), 1.0, 0.0, 3, s,
                          [(0, 0, 0, M - 1, N - 1, 8.0)])
            assert np.array_equal(C, A.astype(np.int64) @ B.astype(np.int64))
            assert rep.corrected == 1 and rep.records[0]["row"] == M - 1


def test_argument_errors(ft, handle):
    import torch
    A = torch.zeros(8, 8, device="cuda")
    with pytest.raises(ft.FtgemmError) as e:
        handle.set_schedule(dict(m_tb=100, n_tb=128, k_tb=8, m_w=32, n_w=64, m_t=8, n_t=8,
                                 cadence=1, split_k=1))
    assert e.value.status == ft.ERR_UNSUPPORTED
    handle.set_schedule(None)
    with pytest.raises(ft.FtgemmError) as e:
        handle.gemm(A, A, A, inject=[(5, 0, 0, 0, 0, 1.0)])
    assert e.value.status == ft.ERR_ARG
    with pytest.raises(ft.FtgemmError) as e:
        handle.gemm(A, A, A, inject=[(0, 0, 99, 0, 0, 1.0)])
    assert e.value.status == ft.ERR_ARG
    with pytest.raises(ft.FtgemmError) as e:
        handle.gemm(A, A, A, level=4)
    assert e.value.status == ft.ERR_UNSUPPORTED


def test_empty_operands_rejected(ft, handle):
    # an empty product is an argument error (M, N or K of 0), raised before
    # any work is enqueued; the handle computes normally afterwards
    import torch
    for M, N, K in ((0, 8, 8), (8, 0, 8), (8, 8, 0)):
        A = torch.zeros(M, K, device="cuda")
        B = torch.zeros(K, N, device="cuda")
        C = torch.zeros(M, N, device="cuda")
        with pytest.raises(ft.FtgemmError) as e:
            handle.gemm(A, B, C)
        assert e.value.status == ft.ERR_ARG
    A = synth.integers((40, 24), 900)
    B = synth.integers((24, 56), 901)
    C = torch.zeros(40, 56, device="cuda")
    rep = handle.gemm(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), C)
    assert rep.detected == 0
    assert np.array_equal(C.cpu().numpy(), A.astype(np.int64) @ B.astype(np.int64))


# ---------------------------------------------------------------------------
# floating-point inputs
# ---------------------------------------------------------------------------

def _float_bound(A, B, Cin, alpha, beta):
    """Componentwise worst-case bound 2*K*u*(|alpha||A||B| + |beta||C_in|)."""
    K = A.shape[1]
    absprod = np.abs(A.astype(np.float64)) @ np.abs(B.astype(np.float64))
    return 2 * K * U32 * (abs(alpha) * absprod + abs(beta) * np.abs(Cin.astype(np.float64)))


@pytest.mark.parametrize("level", ["thread", "warp", "block"])
def test_float_parity_and_faults(ft, handle, orc, level):
    """U(-1,1) inputs, alpha=1, beta=0.5 (the square-sweep workload, reduced):
    C within the worst-case bound, no false alarm, faults of 1e-2..1e3 x the
    tile max located exactly as the oracle does and corrected to within tau."""
    M, N, K = 384, 256, 1024
    A = synth.uniform((M, K), synth.workload_seed("sweep_fp32", 0))
    B = synth.uniform((K, N), synth.workload_seed("sweep_fp32", 1))
    Cin = synth.uniform((M, N), synth.workload_seed("sweep_fp32", 2))
    lv = LEVELS[level]
    s = _sched("huge", cadence=32)
    clean_o = orc.gemm_ft(A, B, _oracle_sched(orc, s, lv), alpha=1.0, beta=0.5, Cin=Cin)
    C0, rep0 = _run(ft, handle, A, B, Cin, 1.0, 0.5, lv, s, [])
    bound = _float_bound(A, B, Cin, 1.0, 0.5)
    assert np.all(np.abs(C0 - clean_o.C) <= bound)
    assert rep0.detected == 0 and clean_o.detected == 0
    # faults: magnitudes log-uniform in [1e-2, 1e3] x the tile's max |A B|
    AB = A.astype(np.float64) @ B.astype(np.float64)
    pos = synth.fault_positions(synth.workload_seed("sweep_fp32", 3), 6, 3, 2, K // 8, 128, 128, M, N, 32,
                                unit_of=_unit_fn(s, lv))
    mags = synth.log_uniform(synth.workload_seed("sweep_fp32", 4), 6, 1e-2, 1e3)
    faults = []
    for (tm, tn, ks, r, c), g in zip(pos, mags):
        tmax = np.abs(AB[tm * 128:(tm + 1) * 128, tn * 128:(tn + 1) * 128]).max()
        faults.append((tm, tn, ks, r, c, float(np.float32(g * tmax))))
    res = orc.gemm_ft(A, B, _oracle_sched(orc, s, lv), faults=faults, alpha=1.0, beta=0.5, Cin=Cin)
    C, rep = _run(ft, handle, A, B, Cin, 1.0, 0.5, lv, s, faults)
    # every fault is far above its threshold here, so the flagged positions are unique
    for o in res.records:
        assert abs(o.delta) > 4 * o.tau
    assert [_key(r) for r in rep.records] == [_key(r) for r in res.records]
    assert rep.corrected == len(faults) == res.corrected
    for g, o in zip(rep.records, res.records):
        assert g["delta"] == pytest.approx(o.delta, abs=o.tau)
    # corrected elements carry the residual's rounding noise (< tau); the rest the usual bound
    slack = np.zeros_like(bound)
    for o in res.records:
        slack[o.row, o.col] = o.tau
    assert np.all(np.abs(C - res.C) <= bound + slack)
