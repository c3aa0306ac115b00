"""Offline (detect-only, recompute) ABFT, Section 5.5: an attempt in which a
fault is detected is discarded and the GEMM recomputed from C_in; the
accepted result is the fault-free product; when every attempt is hit the
call says so."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def _setup(M, N, K, seed):
    import torch
    A = synth.integers((M, K), seed)
    B = synth.integers((K, N), seed + 1)
    Cin = synth.integers((M, N), seed + 2)
    return A, B, Cin, torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()


def test_discards_hit_attempts_and_recomputes_from_c_in(orc):
    import torch
    import paper_2305_01024_gb300 as ft
    M, N, K = 300, 260, 520
    A, B, Cin, dA, dB = _setup(M, N, K, 61)
    h = ft.Handle(0)
    injects = [[(0, 0, 3, 5, 7, 2.0 ** 10)],                      # attempt 1: hit
               [(1, 1, 20, 1, 2, -2.0 ** 9), (2, 0, 30, 9, 9, 64.0)],  # attempt 2: hit twice
               None]                                               # attempt 3: clean
    dC = torch.from_numpy(Cin.copy()).cuda()
    st, runs, rep = h.gemm_offline(dA, dB, dC, alpha=2.0, beta=-1.0, injects=injects, max_runs=5)
    torch.cuda.synchronize()
    assert st == ft.OK and runs == 3
    assert rep.detected == 3  # every hit was seen (the detector verifies once per tile)
    want = orc.gemm_ref(A, B, 2.0, -1.0, Cin)
    assert np.array_equal(dC.cpu().numpy().astype(np.float64), want)
    h.close()


def test_every_attempt_hit_is_unrecovered():
    import torch
    import paper_2305_01024_gb300 as ft
    M, N, K = 256, 256, 256
    _, _, Cin, dA, dB = _setup(M, N, K, 71)
    h = ft.Handle(0)
    injects = [[(0, 1, 2, 3, 4, 2.0 ** 10)], [(1, 0, 5, 6, 7, 2.0 ** 10)]]
    dC = torch.from_numpy(Cin.copy()).cuda()
    st, runs, rep = h.gemm_offline(dA, dB, dC, injects=injects, max_runs=2)
    assert st == ft.ERR_UNRECOVERED and runs == 2 and rep.detected == 2
    assert b"attempts" in ft.lib().ftgemm_last_error()
    h.close()


def test_clean_first_attempt_is_one_run(orc):
    import torch
    import paper_2305_01024_gb300 as ft
    M, N, K = 200, 130, 300
    A, B, Cin, dA, dB = _setup(M, N, K, 81)
    h = ft.Handle(0)
    dC = torch.zeros(M, N, device="cuda")
    st, runs, rep = h.gemm_offline(dA, dB, dC)
    assert st == ft.OK and runs == 1 and rep.detected == 0
    assert np.array_equal(dC.cpu().numpy().astype(np.float64), orc.gemm_ref(A, B))
    h.close()
