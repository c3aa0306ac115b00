"""ftgemm_gemm_noalloc, the entry point for callers that may not allocate
device memory (for example because a framework's memory pool owns the
device, or because cudaMalloc could synchronise the device at a bad time).

It is checked against the ordinary ftgemm_gemm on the same inputs and with
the same schedule (the 128 x 128 x 16 tile, verification every 16 k-steps),
through the C ABI, at every fp32 checksum level, on two calls in a row (the
second call must not be disturbed by what the first left in the shared fixed
array): bit for bit on integer inputs, within the worst-case rounding bound
on float inputs.  Once the first call on the device has done its set-up,
calls leave the device's free memory unchanged.  A problem too large for the
fixed array is refused with a clear message.
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


@pytest.mark.parametrize("level", ["FT_OFF", "FT_THREAD", "FT_WARP", "FT_BLOCK"])
def test_noalloc_matches_gemm_on_two_calls(level):
    import torch
    import paper_2305_01024_gb300 as ft
    lv = getattr(ft, level)
    f = _fn(ft)
    h = ft.Handle(0)
    h.set_schedule(SCHED)
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    cases = [("int", (300, 260, 520), 1.0, 0.0), ("uniform", (257, 390, 1000), 0.75, -0.5)]
    runs = []
    for call, (kind, (M, N, K), alpha, beta) in enumerate(cases):
        A = synth.make(kind, (M, K), 9000 + call)
        B = synth.make(kind, (K, N), 9100 + call)
        Cin = synth.make(kind, (M, N), 9200 + call)
        dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
        ref = torch.from_numpy(Cin.copy()).cuda()
        rep_ref = h.gemm(dA, dB, ref, alpha=alpha, beta=beta, level=lv)
        out = torch.from_numpy(Cin.copy()).cuda()
        recs = (ft.FaultRecord * 16)()
        runs.append((kind, A, B, Cin, alpha, beta, dA, dB, ref, rep_ref, out, recs, ft.Report(capacity=16, records=recs)))
    # the first call on the device may do its set-up (and allocate); make it
    # on a separate output
    warm = torch.zeros(8, 8, device="cuda")
    z = torch.zeros(8, 8, device="cuda")
    assert f(8, 8, 8, 1.0, z.data_ptr(), 8, z.data_ptr(), 8, 0.0, warm.data_ptr(), 8, lv, stream, None) == 0
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for kind, A, B, Cin, alpha, beta, dA, dB, ref, rep_ref, out, recs, rep in runs:
        M, K = A.shape
        N = B.shape[1]
        rc = f(M, N, K, alpha, dA.data_ptr(), K, dB.data_ptr(), N, beta, out.data_ptr(), N, lv, stream,
               C.byref(rep))
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
        assert rep.detected == rep_ref.detected == 0 and rep.n_records == 0 and not rep.overflow
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0, "a call after the set-up changed the device's free memory"
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
