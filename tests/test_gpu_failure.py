"""Failure detection without a GPU fault: a device wait that nothing
satisfies gives up after its limit, the kernel returns, the host reads
FTGEMM_ERR_TIMEOUT, and the context stays usable (a GEMM right after it is
exact)."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def test_bounded_wait_gives_up_and_the_handle_survives(orc):
    import torch
    import paper_2305_01024_gb300 as ft
    L = ft.lib()
    h = ft.Handle(0)
    rc = L.ftgemm_selftest_wait(h._h, 1 << 21)  # about a millisecond
    assert rc == ft.ERR_TIMEOUT
    assert b"gave up" in L.ftgemm_last_error()
    # the report was cleared by the fetch: the next call is clean
    M, N, K = 200, 300, 136
    A = synth.integers((M, K), 77)
    B = synth.integers((K, N), 78)
    dC = torch.zeros(M, N, device="cuda")
    rep = h.gemm(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), dC, level=ft.FT_BLOCK)
    torch.cuda.synchronize()
    assert rep.detected == 0
    assert np.array_equal(dC.cpu().numpy().astype(np.float64), orc.gemm_ref(A, B))
    h.close()
