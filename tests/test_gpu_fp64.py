"""Double and double-complex GEMM with online block-level ABFT (Section 6:
the DGEMM / ZGEMM extension) through the C ABI, against the oracle.

Integer and Gaussian-integer inputs make every product and sum exact, so C
and the fault records must equal the oracle's bit for bit; float inputs are
compared within the rounding bound, with the corrected elements allowed their
threshold."""
import ctypes as C
import math

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu
U64 = 2.0 ** -53


@pytest.fixture(scope="module")
def ft():
    import torch
    import paper_2305_01024_gb300 as ft
    assert torch.cuda.is_available()
    ft.lib()
    return ft


def _key(r):
    if isinstance(r, dict):
        return (r["tile_m"], r["tile_n"], r["kstep"], r["row"], r["col"], r["kind"])
    return (r.tile_m, r.tile_n, r.kstep, r.row, r.col, r.kind)


def _ints(shape, seed):
    return synth.integers(shape, seed, dtype=np.float64)


def _cints(shape, seed):
    return _ints(shape, seed) + 1j * _ints(shape, seed + 7919)


def _cuda(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _f32(d):
    """Deltas travel as float32 through the injection spec: give the oracle the same value."""
    return float(np.float32(d))


# ---- DGEMM -------------------------------------------------------------------

@pytest.mark.parametrize("cadence", [1, 4, 0])
def test_dgemm_integers_bit_exact_every_target(ft, orc, cadence):
    M, N, K = 300, 260, 520  # ragged 128 x 128 tiles, 65 k-steps of 8
    A, B, Cin = _ints((M, K), 101), _ints((K, N), 102), _ints((M, N), 103)
    faults = [(0, 0, 2, 5, 7, 64.0), (2, 1, 60, 40, 3, -128.0), (1, 2, 31, 9, 2, 32.0),
              (1, 0, 10, 4, 4, 16.0, 1), (0, 1, 12, 6, 8, 16.0, 2), (2, 2, -1, 43, 3, 2.0 ** 20)]
    h = ft.Handle(0)
    dC = _cuda(Cin)
    rep = h.dgemm(_cuda(A), _cuda(B), dC, alpha=2.0, beta=-1.0, cadence=cadence, inject=faults)
    sched = orc.dgemm_schedule(cadence=cadence if cadence > 0 else 65)
    res = orc.gemm_ft(A, B, sched, faults=faults, alpha=2.0, beta=-1.0, Cin=Cin)
    assert np.array_equal(dC.cpu().numpy(), res.C)
    assert sorted(map(_key, rep.records)) == sorted(map(_key, res.records))
    mine = {_key(r): r for r in rep.records}
    for r in res.records:
        g = mine[_key(r)]
        assert g["delta"] == r.delta and g["residual_r"] == r.residual_r and g["residual_c"] == r.residual_c
        assert g["tau"] == pytest.approx(r.tau, rel=1e-12)
    assert rep.corrected == res.corrected and rep.checksum_only == res.checksum_only
    h.close()


def test_dgemm_float_inputs_match_the_oracle(ft, orc):
    M, N, K = 384, 256, 1000
    A = synth.normal((M, K), 111).astype(np.float64)
    B = synth.normal((K, N), 112).astype(np.float64)
    pos = synth.fault_positions(113, 5, 3, 2, 125, 128, 128, M, N, 16)
    faults = [(a, b, ks, r, c, _f32(1e-9 * math.sqrt(K) * (2 + q))) for q, (a, b, ks, r, c) in enumerate(pos)]
    h = ft.Handle(0)
    dC = _cuda(np.zeros((M, N)))
    rep = h.dgemm(_cuda(A), _cuda(B), dC, cadence=16, inject=faults)
    res = orc.gemm_ft(A, B, orc.dgemm_schedule(cadence=16), faults=faults)
    assert sorted(map(_key, rep.records)) == sorted(map(_key, res.records))
    assert rep.corrected == 5
    got = dC.cpu().numpy()
    exact = A @ B
    bound = 2 * K * U64 * (np.abs(A) @ np.abs(B))
    slack = np.zeros_like(got)
    for r in rep.records:
        slack[r["row"], r["col"]] = r["tau"]
    assert np.all(np.abs(got - exact) <= bound + slack)
    h.close()


def test_dgemm_off_keeps_faults_and_checks_nothing(ft, orc):
    M, N, K = 200, 140, 96
    A, B = _ints((M, K), 121), _ints((K, N), 122)
    h = ft.Handle(0)
    dC = _cuda(np.zeros((M, N)))
    rep = h.dgemm(_cuda(A), _cuda(B), dC, level=ft.FT_OFF, inject=[(1, 0, 3, 10, 20, 8.0)])
    want = A @ B
    want[128 + 10, 20] += 8.0
    assert np.array_equal(dC.cpu().numpy(), want) and rep.detected == 0
    with pytest.raises(ft.FtgemmError) as e:
        h.dgemm(_cuda(A), _cuda(B), dC, level=ft.FT_OFF, inject=[(1, 0, 3, 10, 20, 8.0, 1)])
    assert e.value.status == ft.ERR_ARG
    with pytest.raises(ft.FtgemmError) as e:
        h.dgemm(_cuda(A), _cuda(B), dC, level=ft.FT_THREAD)
    assert e.value.status == ft.ERR_UNSUPPORTED
    h.close()


def test_dgemm_no_false_alarm_on_normal_data(ft):
    import torch
    n = 1536
    A = synth.torch_make("normal", (n, n), 131, "cuda", torch.float64)
    B = synth.torch_make("normal", (n, n), 132, "cuda", torch.float64)
    C_ = torch.empty(n, n, dtype=torch.float64, device="cuda")
    h = ft.Handle(0)
    rep = h.dgemm(A, B, C_, cadence=1)
    assert rep.detected == 0
    ref = A @ B
    assert torch.allclose(C_, ref, rtol=0, atol=float(4 * n * U64 * (A.abs() @ B.abs()).max()))
    h.close()


def test_dgemm_full_size_sampled_rows(ft, orc):
    """The bench's DGEMM workload: 4096^3, N(0,1), block level, cadence 16;
    every fault located and corrected, sampled rows against the oracle."""
    import torch
    n = 4096
    A = synth.torch_make("normal", (n, n), synth.workload_seed("dgemm", 0), "cuda", torch.float64)
    B = synth.torch_make("normal", (n, n), synth.workload_seed("dgemm", 1), "cuda", torch.float64)
    tiles, ks = n // 128, n // 8
    pos = synth.fault_positions(synth.workload_seed("dgemm", 2), 8, tiles, tiles, ks, 128, 128, n, n, 16)
    faults = [(a, b, k, r, c, _f32(1e-8 * math.sqrt(n))) for (a, b, k, r, c) in pos]
    h = ft.Handle(0)
    C_ = torch.empty(n, n, dtype=torch.float64, device="cuda")
    rep = h.dgemm(A, B, C_, cadence=16, inject=faults)
    where = [(a * 128 + r, b * 128 + c) for (a, b, k, r, c, d) in faults]
    assert sorted((x["row"], x["col"], x["kind"]) for x in rep.records) == sorted((i, j, 0) for i, j in where)
    rows = sorted(set(int(u * n) for u in synth.unit(synth.workload_seed("dgemm", 3), 8)) | {i for i, _ in where})
    Ar, Bh = A[rows].cpu().numpy(), B.cpu().numpy()
    ref = orc.gemm_ref(Ar, Bh)
    got = C_[rows].cpu().numpy()
    bound = 2 * n * U64 * (np.abs(Ar) @ np.abs(Bh))
    slack = np.zeros_like(got)
    for x in rep.records:
        slack[rows.index(x["row"]), x["col"]] = x["tau"]
    assert np.all(np.abs(got - ref) <= bound + slack)
    h.close()


# ---- ZGEMM -------------------------------------------------------------------

def _zkey_res(r):
    return (r.tile_m, r.tile_n, r.kstep, r.row, r.col, r.kind)


@pytest.mark.parametrize("cadence", [1, 3])
def test_zgemm_gaussian_integers_bit_exact(ft, orc, cadence):
    M, N, K = 150, 140, 200  # ragged 64 x 64 tiles, 25 k-steps
    A, B, Cin = _cints((M, K), 201), _cints((K, N), 202), _cints((M, N), 203)
    I = ft.TARGET_IMAG
    faults = [(0, 0, 2, 5, 7, 64.0), (2, 1, 24, 21, 3, -128.0, I), (1, 2, 11, 9, 2, 32.0, 1 | I),
              (1, 0, 10, 4, 4, 16.0, 1), (0, 1, 12, 6, 8, 16.0, 2 | I), (2, 2, -1, 21, 11, 2.0 ** 20, I)]
    alpha, beta = 2 - 1j, 0.5 + 1j
    h = ft.Handle(0)
    dC = _cuda(Cin)
    rep = h.zgemm(_cuda(A), _cuda(B), dC, alpha=alpha, beta=beta, cadence=cadence, inject=faults)
    res = orc.zgemm_ft(A, B, tile=64, k_tb=8, cadence=cadence, faults=faults, alpha=alpha, beta=beta, Cin=Cin)
    assert np.array_equal(dC.cpu().numpy(), res.C)
    assert sorted(map(_key, rep.records)) == sorted(map(_zkey_res, res.records))
    mine = {_key(r): r for r in rep.records}
    for r in res.records:
        g = mine[_zkey_res(r)]
        assert g["delta"] == r.delta and g["residual_r"] == r.residual_r and g["residual_c"] == r.residual_c
        assert g["tau"] == pytest.approx(r.tau, rel=1e-12)
    h.close()


def test_zgemm_float_inputs_match_the_oracle(ft, orc):
    M, N, K = 200, 130, 400
    A = synth.normal((M, K), 211).astype(np.float64) + 1j * synth.normal((M, K), 212).astype(np.float64)
    B = synth.normal((K, N), 213).astype(np.float64) + 1j * synth.normal((K, N), 214).astype(np.float64)
    pos = synth.fault_positions(215, 4, 4, 3, 50, 64, 64, M, N, 4)
    faults = [(a, b, ks, r, c, _f32(1e-9 * math.sqrt(K) * (3 + q)), ft.TARGET_IMAG * (q % 2))
              for q, (a, b, ks, r, c) in enumerate(pos)]
    h = ft.Handle(0)
    dC = _cuda(np.zeros((M, N), np.complex128))
    rep = h.zgemm(_cuda(A), _cuda(B), dC, cadence=4, inject=faults)
    res = orc.zgemm_ft(A, B, tile=64, k_tb=8, cadence=4, faults=faults)
    assert sorted(map(_key, rep.records)) == sorted(map(_zkey_res, res.records))
    assert rep.corrected == 4
    got = dC.cpu().numpy()
    exact = A @ B
    bound = 4 * K * U64 * (np.abs(A) @ np.abs(B))
    slack = np.zeros(got.shape)
    for r in rep.records:
        slack[r["row"], r["col"]] = r["tau"]
    assert np.all(np.abs(got - exact) <= bound + slack)
    h.close()


def test_zgemm_alignment_is_checked(ft):
    import torch
    h = ft.Handle(0)
    buf = torch.zeros(2 * 64 * 64 + 1, dtype=torch.float64, device="cuda")
    one = (C.c_double * 2)(1.0, 0.0)
    L = ft.lib()
    p = C.c_void_p(buf.data_ptr() + 8)  # 8-byte aligned, not 16
    st = L.ftgemm_zgemm(h._h, 8, 8, 8, one, p, 8, p, 8, one, p, 8, ft.FT_BLOCK, 1, None, None, None)
    assert st == ft.ERR_ALIGN
    h.close()


@pytest.mark.parametrize("shape", [(1, 1, 1), (1, 300, 7), (129, 1, 9), (65, 70, 13)])
def test_fp64_degenerate_and_ragged_shapes(ft, orc, shape):
    """One element, one row or column, K not a multiple of the k-step: both
    kernels against the oracle, bit-exact on integers, with a fault each."""
    M, N, K = shape
    A, B = _ints((M, K), 301 + M), _ints((K, N), 302 + N)

    def last(T, target):  # a fault on the last element, in tile coordinates of tile size T
        return [((M - 1) // T, (N - 1) // T, 0, (M - 1) % T, (N - 1) % T, 8.0, target)]

    fd = last(ft.DGEMM_TILE, 0)
    h = ft.Handle(0)
    dC = _cuda(np.zeros((M, N)))
    rep = h.dgemm(_cuda(A), _cuda(B), dC, cadence=1, inject=fd)
    res = orc.gemm_ft(A, B, orc.dgemm_schedule(cadence=1), faults=fd)
    assert np.array_equal(dC.cpu().numpy(), res.C)
    assert sorted(map(_key, rep.records)) == sorted(map(_key, res.records))
    Z, W = A + 1j * _ints((M, K), 303), B - 1j * _ints((K, N), 304)
    fz = last(ft.ZGEMM_TILE, ft.TARGET_IMAG)
    dZ = _cuda(np.zeros((M, N), np.complex128))
    rz = h.zgemm(_cuda(Z), _cuda(W), dZ, cadence=1, inject=fz)
    oz = orc.zgemm_ft(Z, W, tile=64, k_tb=8, cadence=1, faults=fz)
    assert np.array_equal(dZ.cpu().numpy(), oz.C)
    assert sorted(map(_key, rz.records)) == sorted(map(_zkey_res, oz.records))
    h.close()
