"""The autotuners.  The fp32 one on the irregular FP32 shapes of the paper's evaluation
(tall-skinny, small-K, long-K, unaligned), each with one seeded fault, at
full size.  C is checked against the oracle on sampled rows (every row the
fault touches among them); the fault is located and corrected.  The
tensor-core ones (single CTAs or CTA pairs) on a GEMM and on a group, whose
results stay exact on integer inputs whichever schedule they pick."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu
U32 = 2.0 ** -24
SHAPES = [(16384, 16384, 32), (20480, 256, 20480), (256, 256, 65536), (4096, 96, 4096), (777, 1531, 2049)]
TUPLES = {(128, 128, 16, 64, 64, 16, 8), (128, 128, 32, 64, 64, 16, 8), (128, 128, 16, 32, 64, 8, 8), (128, 128, 8, 32, 64, 8, 8),
          (64, 64, 8, 32, 64, 8, 8), (32, 128, 8, 16, 64, 4, 8), (32, 32, 8, 16, 32, 4, 4),
          (16, 16, 16, 8, 16, 2, 2)}


@pytest.fixture(scope="module")
def ft():
    import torch
    import paper_2305_01024_gb300 as ft
    assert torch.cuda.is_available()
    ft.lib()
    return ft


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "x".join(map(str, s)))
def test_autotuned_irregular_shape_one_fault(ft, orc, shape):
    import torch
    M, N, K = shape
    q = SHAPES.index(shape)
    h = ft.Handle(0)
    A = synth.torch_make("normal", (M, K), synth.workload_seed("irregular_fp32", 2 * q), "cuda")
    B = synth.torch_make("normal", (K, N), synth.workload_seed("irregular_fp32", 2 * q + 1), "cuda")
    C = torch.empty(M, N, device="cuda")
    s, lv = h.autotune(A, B, C, level=ft.FT_AUTO, reps=2)
    assert lv in (ft.FT_THREAD, ft.FT_WARP, ft.FT_BLOCK)
    assert (s.m_tb, s.n_tb, s.k_tb, s.m_w, s.n_w, s.m_t, s.n_t) in TUPLES and s.split_k >= 1
    # the tuned schedule is what the handle now uses for this shape
    g = h.get_schedule(M, N, K, ft.F32, ft.FT_AUTO)
    assert g.as_dict() == s.as_dict()
    # one seeded fault on the tuned tiling
    tiles_m, tiles_n = -(-M // s.m_tb), -(-N // s.n_tb)
    ksteps = -(-K // s.k_tb)
    (tm, tn, ks, r, c), = synth.fault_positions(synth.workload_seed("irregular_fp32", 50 + q), 1, tiles_m, tiles_n, ksteps,
                                                s.m_tb, s.n_tb, M, N, max(1, s.cadence))
    delta = 64.0 * np.sqrt(K)
    C.zero_()
    rep = h.gemm(A, B, C, level=ft.FT_AUTO, inject=[(tm, tn, ks, r, c, delta)])
    torch.cuda.synchronize()
    i, j = tm * s.m_tb + r, tn * s.n_tb + c
    assert [(x["row"], x["col"], x["kind"]) for x in rep.records] == [(i, j, 0)]
    sample = [int(u * M) for u in synth.unit(synth.workload_seed("irregular_fp32", 60 + q), 32)]
    rows = sorted(set([i] + sample) | set(range(min(M, 8))))
    Ar = A[rows].cpu().numpy()
    Bh = B.cpu().numpy()
    ref = orc.gemm_ref(Ar, Bh)
    got = C[rows].cpu().numpy().astype(np.float64)
    bound = 2 * K * U32 * (np.abs(Ar.astype(np.float64)) @ np.abs(Bh.astype(np.float64)))
    slack = np.zeros_like(got)
    slack[rows.index(i), j] = rep.records[0]["tau"]  # the corrected value carries the threshold
    assert np.all(np.abs(got - ref) <= bound + slack)
    h.close()


# ---- tensor-core schedules: single CTAs or CTA pairs, by measurement -------

def _int_bf16(shape, seed):
    import torch
    x = synth.integers(shape, seed).astype(np.float32)
    return x, torch.from_numpy(x).cuda().to(torch.bfloat16)


@pytest.mark.parametrize("level", ["off", "tile"])
def test_tc_autotune_picks_a_schedule_and_keeps_results_exact(ft, level):
    """ftgemm_autotune_tc times both schedules on the operands and caches the
    faster for the shape; calls of that shape then run on it, and stay
    exact on integer inputs whichever it is."""
    import torch
    M, N, K = 1000, 1536, 520
    A, dA = _int_bf16((M, K), 7100)
    B, dB = _int_bf16((K, N), 7101)
    h = ft.Handle(0)
    C = torch.empty(M, N, device="cuda")
    pick = h.autotune_tc(dA, dB, C, level=ft.LEVELS[level], dtype=ft.BF16, reps=2)
    assert isinstance(pick, bool)
    ref = A.astype(np.int64) @ B.astype(np.int64)
    assert np.array_equal(C.cpu().numpy().astype(np.int64), ref)  # the last timed call
    C.zero_()
    rep = h.gemm(dA, dB, C, level=ft.LEVELS[level], dtype=ft.BF16)
    assert np.array_equal(C.cpu().numpy().astype(np.int64), ref) and rep.detected == 0
    with pytest.raises(ft.FtgemmError):
        h.autotune_tc(dA, dB, C, level=ft.FT_BLOCK, dtype=ft.BF16)
    h.close()


def test_group_autotune_returns_the_faster_schedule(ft):
    import torch
    shapes = [(300, 500, 256), (1000, 260, 640), (64, 64, 64), (777, 1248, 1008)]
    h = ft.Handle(0)
    host, probs = [], []
    for q, (M, N, K) in enumerate(shapes):
        A, dA = _int_bf16((M, K), 7200 + 2 * q)
        B, dB = _int_bf16((K, N), 7201 + 2 * q)
        host.append((A, B))
        probs.append((dA, dB, torch.empty(M, N, device="cuda")))
    g = ft.Group(h, probs, dtype=ft.BF16, level=ft.FT_TILE, tune=2)
    assert g.pair in (True, False)
    for pr in probs:
        pr[2].zero_()
    g.run()
    torch.cuda.synchronize()
    assert h.report_fetch().detected == 0
    for (A, B), pr in zip(host, probs):
        assert np.array_equal(pr[2].cpu().numpy().astype(np.int64), A.astype(np.int64) @ B.astype(np.int64))
    g.close()
    h.close()
