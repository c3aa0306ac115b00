"""The non-fused ABFT baseline (Section 5.3's comparison scheme: rank-K_s
updates, separate checksum GEMMs and a separate verification kernel) against
the oracle run at block level with cadence K_s / 16, and against the fused
kernel on the same faults."""
import ctypes as C

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
    L = ft.lib()
    L.ftgemm_gemm_nonfused.argtypes = [C.c_void_p, C.c_int64, C.c_int64, C.c_int64, C.c_double, C.c_void_p,
                                       C.c_int64, C.c_void_p, C.c_int64, C.c_double, C.c_void_p, C.c_int64,
                                       C.c_int32, C.POINTER(ft.InjectSpec), C.POINTER(ft.Report)]
    L.ftgemm_gemm_nonfused.restype = C.c_int
    return ft


def _nonfused(ft, h, A, B, Cin, alpha, beta, ks, faults):
    import torch
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    dC = torch.from_numpy(Cin.copy()).cuda()
    M, K = A.shape
    N = B.shape[1]
    spec = ft.make_inject(faults) if faults else None
    recs = (ft.FaultRecord * 4096)()
    rep = ft.Report(capacity=4096, records=recs)
    rc = ft.lib().ftgemm_gemm_nonfused(h._h, M, N, K, alpha, dA.data_ptr(), K, dB.data_ptr(), N, beta,
                                       dC.data_ptr(), N, ks, C.byref(spec) if spec else None, C.byref(rep))
    assert rc == 0, ft.lib().ftgemm_last_error()
    torch.cuda.synchronize()
    return dC.cpu().numpy().astype(np.float64), ft._records(rep, 4096), rep


def _sched(orc, ks):
    return orc.Schedule(m_tb=128, n_tb=128, k_tb=16, m_w=64, n_w=64, m_t=16, n_t=8, cadence=ks // 16,
                        split_k=1, level=orc.BLOCK, lam=32.0, u=U32)


def _key(r):
    if isinstance(r, dict):
        return (r["tile_m"], r["tile_n"], r["kstep"], r["row"], r["col"], r["kind"])
    return (r.tile_m, r.tile_n, r.kstep, r.row, r.col, r.kind)


def test_int256_integers_bit_exact(ft, orc):
    M = N = K = 256
    A = synth.integers((M, K), synth.workload_seed("int256", 0))
    B = synth.integers((K, N), synth.workload_seed("int256", 1))
    pos = synth.fault_positions(synth.workload_seed("int256", 2), 4, 2, 2, 16, 128, 128, M, N, 16)
    faults = [(tm, tn, ks, r, c, 2.0 ** 10) for (tm, tn, ks, r, c) in pos]
    h = ft.Handle(0)
    got, recs, rep = _nonfused(ft, h, A, B, np.zeros((M, N), np.float32), 1.0, 0.0, 256, faults)
    res = orc.gemm_ft(A, B, _sched(orc, 256), faults=faults)
    assert np.array_equal(got, res.C)
    assert sorted(map(_key, recs)) == sorted(map(_key, res.records))
    assert rep.corrected == 4
    h.close()


@pytest.mark.parametrize("ks", [64, 256])
def test_ragged_alpha_beta_faults_on_every_target(ft, orc, ks):
    M, N, K = 300, 260, 520
    A = synth.integers((M, K), 41)
    B = synth.integers((K, N), 42)
    Cin = synth.integers((M, N), 43)
    faults = [(0, 0, 2, 5, 7, 64.0), (2, 1, 20, 40, 3, -128.0), (1, 2, 31, 9, 2, 32.0),
              (1, 0, 10, 4, 4, 16.0, 1), (0, 1, 12, 6, 8, 16.0, 2)]
    h = ft.Handle(0)
    got, recs, _ = _nonfused(ft, h, A, B, Cin, 2.0, -1.0, ks, faults)
    res = orc.gemm_ft(A, B, _sched(orc, ks), faults=faults, alpha=2.0, beta=-1.0, Cin=Cin)
    assert np.array_equal(got, res.C)
    assert sorted(map(_key, recs)) == sorted(map(_key, res.records))
    h.close()


def test_float_inputs_same_records_as_the_fused_kernel(ft, orc):
    import torch
    M, N, K = 512, 384, 1024
    A = synth.uniform((M, K), 51)
    B = synth.uniform((K, N), 52)
    faults = [(1, 2, 7, 17, 33, 5.0), (3, 0, 40, 100, 1, -7.0), (0, 1, 63, 0, 127, 3.0)]
    h = ft.Handle(0)
    got, recs, _ = _nonfused(ft, h, A, B, np.zeros((M, N), np.float32), 1.0, 0.0, 256, faults)
    h.set_schedule(dict(m_tb=128, n_tb=128, k_tb=16, m_w=64, n_w=64, m_t=16, n_t=8, cadence=16, split_k=1))
    dC = torch.zeros(M, N, device="cuda")
    rep = h.gemm(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), dC, level=ft.FT_BLOCK, inject=faults)
    torch.cuda.synchronize()
    fused = dC.cpu().numpy().astype(np.float64)
    assert sorted((r["row"], r["col"], r["kind"]) for r in recs) == \
        sorted((r["row"], r["col"], r["kind"]) for r in rep.records)
    exact = A.astype(np.float64) @ B.astype(np.float64)
    bound = 2 * K * U32 * (np.abs(A.astype(np.float64)) @ np.abs(B.astype(np.float64)))
    slack = np.zeros_like(exact)
    for r in recs:
        slack[r["row"], r["col"]] = r["tau"]
    assert np.all(np.abs(got - exact) <= bound + slack)
    assert np.all(np.abs(fused - exact) <= bound + slack)
    h.close()
