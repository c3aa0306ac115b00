"""ftgemm_gemm_noalloc, the entry point for callers that may not allocate
device memory (for example because a framework's memory pool owns the
device, or because cudaMalloc could synchronise the device at a bad time).

It is checked against the ordinary ftgemm_gemm on the same inputs, through
the C ABI, on two calls in a row (the second call must not be disturbed by
what the first left in the shared fixed array), and a problem too large for
the fixed array must be refused with a clear message.
"""
import ctypes as C

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24
SCHED = dict(m_tb=128, n_tb=128, k_tb=16, m_w=32, n_w=64, m_t=8, n_t=8, cadence=16, split_k=1)


def _fn(ft):
    L = ft.lib()
    f = L.ftgemm_gemm_noalloc
    i64, vp = C.c_int64, C.c_void_p
    f.argtypes = [i64, i64, i64, C.c_double, vp, i64, vp, i64, C.c_double, vp, i64, C.c_int, vp,
                  C.POINTER(ft.Report)]
    f.restype = C.c_int
    return f


def _bound(A, B, Cin, alpha, beta):
    K = A.shape[1]
    absprod = np.abs(A.astype(np.float64)) @ np.abs(B.astype(np.float64))
    return 2 * K * U32 * (abs(alpha) * absprod + abs(beta) * np.abs(Cin.astype(np.float64)))


def test_noalloc_matches_gemm_on_two_calls():
    import torch
    import paper_2305_01024_gb300 as ft
    f = _fn(ft)
    h = ft.Handle(0)
    h.set_schedule(SCHED)
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    cases = [("int", (300, 260, 520), 1.0, 0.0), ("uniform", (257, 390, 1000), 0.75, -0.5)]
    for call, (kind, (M, N, K), alpha, beta) in enumerate(cases):
        A = synth.make(kind, (M, K), 9000 + call)
        B = synth.make(kind, (K, N), 9100 + call)
        Cin = synth.make(kind, (M, N), 9200 + call)
        dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
        ref = torch.from_numpy(Cin.copy()).cuda()
        rep_ref = h.gemm(dA, dB, ref, alpha=alpha, beta=beta, level=ft.FT_BLOCK)
        out = torch.from_numpy(Cin.copy()).cuda()
        recs = (ft.FaultRecord * 16)()
        rep = ft.Report(capacity=16, records=recs)
        rc = f(M, N, K, alpha, dA.data_ptr(), K, dB.data_ptr(), N, beta, out.data_ptr(), N,
               ft.FT_BLOCK, stream, C.byref(rep))
        assert rc == 0, ft.lib().ftgemm_last_error()
        torch.cuda.synchronize()
        got, want = out.cpu().numpy().astype(np.float64), ref.cpu().numpy().astype(np.float64)
        if kind == "int":
            assert np.array_equal(got, want)
        else:
            exact = alpha * (A.astype(np.float64) @ B.astype(np.float64)) + beta * Cin
            bound = _bound(A, B, Cin, alpha, beta)
            assert np.all(np.abs(got - want) <= bound)
            assert np.all(np.abs(got - exact) <= bound)
        assert rep.detected == rep_ref.detected == 0
    h.close()


def test_noalloc_refuses_a_problem_larger_than_its_array():
    import torch
    import paper_2305_01024_gb300 as ft
    f = _fn(ft)
    n = 4096  # the transposed A alone needs 64 MiB
    A = torch.zeros(n, n, device="cuda")
    rc = f(n, n, n, 1.0, A.data_ptr(), n, A.data_ptr(), n, 0.0, A.data_ptr(), n, ft.FT_BLOCK,
           None, None)
    assert rc == ft.ERR_ARG
    msg = ft.lib().ftgemm_last_error().decode()
    assert "bytes of scratch" in msg
