"""Offline (detect-only, recompute) ABFT, Section 5.5: an attempt in which a
fault is detected is discarded and the GEMM recomputed from C_in; the
accepted result is the fault-free product; when every attempt is hit the
call says so.  The detector (column checksums only, one verification, no
correction) reports what the oracle's detect-only level reports."""
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
               [(1, 1, 10, 1, 2, -2.0 ** 9), (2, 0, 15, 9, 9, 64.0)],  # attempt 2: hit twice
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


def test_detector_matches_oracle_detect_level(orc):
    """One attempt over integer inputs with offsets in five tiles (one of
    them on a column checksum, one on a row checksum, which the detector does
    not keep): the detections equal the oracle's detect-only level, record
    for record, residuals exact; C keeps the offsets on the accumulator."""
    import torch
    import paper_2305_01024_gb300 as ft
    M, N, K = 384, 300, 700
    A, B, _, dA, dB = _setup(M, N, K, 91)
    nks = -(-K // 32)
    faults = [(0, 0, 2, 5, 7, 2.0 ** 10), (1, 1, 21, 100, 33, -256.0), (2, 2, 0, 127, 43, 64.0),
              (0, 2, 11, 3, 4, 512.0, 2), (2, 0, 11, 3, 4, 512.0, 1)]
    h = ft.Handle(0)
    dC = torch.zeros(M, N, device="cuda")
    st, runs, rep = h.gemm_offline(dA, dB, dC, injects=[faults], max_runs=1)
    h.close()
    assert st == ft.ERR_UNRECOVERED and runs == 1
    res = orc.gemm_ft(A, B, orc.Schedule(m_tb=128, n_tb=128, k_tb=32, m_w=64, n_w=64, m_t=16, n_t=8,
                                         cadence=nks, level=orc.DETECT), faults=faults)
    got = sorted((x["tile_m"], x["tile_n"], x["kstep"], x["row"], x["col"], x["kind"], x["residual_c"])
                 for x in rep.records)
    want = sorted((x.tile_m, x.tile_n, x.kstep, x.row, x.col, x.kind, x.residual_c) for x in res.records)
    assert got == want and len(got) == 4
    assert np.array_equal(dC.cpu().numpy().astype(np.float64), res.C)


@pytest.mark.parametrize("kind", ["uniform", "positive"])
def test_detector_no_false_alarm_on_float_inputs(kind):
    import torch
    import paper_2305_01024_gb300 as ft
    M = N = 1024
    K = 8192
    A = synth.uniform((M, K), 95)
    B = synth.uniform((K, N), 96)
    if kind == "positive":
        A, B = (A + 1) / 2, (B + 1) / 2
    h = ft.Handle(0)
    dC = torch.zeros(M, N, device="cuda")
    st, runs, rep = h.gemm_offline(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), dC)
    h.close()
    assert st == ft.OK and runs == 1 and rep.detected == 0
