"""Parity at the workloads' full sizes, in the launch configurations bench.py
times, on outputs the oracle computes one by one: sampled rows of C (every
row holding a fault among them), and every fault located and corrected.

* the fp32 headline: 16384^3 fp32, block-level checksums on the 128 x 128 tile with
  16 x 8 fragments and k-steps of 32, verification every 256 of K, alpha 1,
  beta 0.5;
* the tensor-core square: 16384^3 bf16 and e4m3, tile-level checksums through the tensor
  cores (e4m3: the quantizer against the oracle's on sampled rows);
* the 512-problem bf16 group, one persistent launch, 1% of tiles
  faulted; sampled problems compared in full.
"""
import math

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu
U32 = 2.0 ** -24
# Statistical float tolerance: an fp32 dot product of length K rounds with an
# error whose typical size is u*sqrt(K)*|a||b| or below (random rounding
# errors add like a random walk); a corrected element adds the rounding noise
# of its row residual, far smaller.  A dropped k-slice of 32 terms moves an
# element by about sqrt(32) |a||b|/K, i.e. 40 or more of these units at
# K = 16384, so the check below catches it where the worst-case 2Ku bound
# (about 10^4 times looser) does not.
STAT_C = 8.0
# data tile of the tensor-core path with checksums (ftgemm_tc_tile)
TDM_BF16, TDN_BF16, TDM_E4M3, TDN_E4M3 = 125, 252, 123, 248


def _stat_check(got, ref, Ar, Bh, K, cin_abs=None, scale=1.0):
    """max |C - C_ref| / (u sqrt(K) ||a_i|| ||b_j|| * scale + 2u |C_ref|) <= STAT_C."""
    na = np.sqrt((np.asarray(Ar, np.float64) ** 2).sum(1))
    nb = np.sqrt((np.asarray(Bh, np.float64) ** 2).sum(0))
    unit = U32 * math.sqrt(K) * np.outer(na, nb) * scale + 2 * U32 * np.abs(ref)
    if cin_abs is not None:
        unit = unit + 2 * U32 * cin_abs
    ratio = np.abs(got - ref) / unit
    assert ratio.max() <= STAT_C, f"max error {ratio.max():.3g} units of u sqrt(K)|a||b|"
    return float(ratio.max())


@pytest.fixture(scope="module")
def ft():
    import torch
    import paper_2305_01024_gb300 as ft
    assert torch.cuda.is_available()
    ft.lib()
    return ft


def _rows(seed, M, extra):
    return sorted(set(int(u * M) for u in synth.unit(seed, 12)) | set(extra))


def test_fp32_block_16384_sampled_rows(ft, orc):
    import torch
    n = 16384
    sched = dict(m_tb=128, n_tb=128, k_tb=32, m_w=64, n_w=64, m_t=16, n_t=8, cadence=8, split_k=1)
    A = synth.torch_make("uniform", (n, n), synth.workload_seed("sweep_fp32", 0), "cuda")
    B = synth.torch_make("uniform", (n, n), synth.workload_seed("sweep_fp32", 1), "cuda")
    C0 = synth.torch_make("uniform", (n, n), synth.workload_seed("sweep_fp32", 2), "cuda")
    tiles, ksteps = n // 128, n // 32
    pos = synth.fault_positions(synth.workload_seed("sweep_fp32", 70), 6, tiles, tiles, ksteps, 128, 128, n, n, 8)
    mags = synth.log_uniform(synth.workload_seed("sweep_fp32", 71), 6, 1e-1, 1e3)
    faults = [(tm, tn, ks, r, c, float(g * 4 * math.sqrt(n / 9))) for (tm, tn, ks, r, c), g in zip(pos, mags)]
    h = ft.Handle(0)
    h.set_schedule(sched)
    C = C0.clone()
    rep = h.gemm(A, B, C, alpha=1.0, beta=0.5, level=ft.FT_BLOCK, inject=faults)
    torch.cuda.synchronize()
    where = [(tm * 128 + r, tn * 128 + c) for (tm, tn, ks, r, c, d) in faults]
    assert sorted((x["row"], x["col"], x["kind"]) for x in rep.records) == sorted((i, j, 0) for i, j in where)
    rows = _rows(synth.workload_seed("sweep_fp32", 72), n, [i for i, _ in where])
    Ar, Bh, Cr = A[rows].cpu().numpy(), B.cpu().numpy(), C0[rows].cpu().numpy()
    ref = orc.gemm_ref(Ar, Bh, 1.0, 0.5, Cr)
    got = C[rows].cpu().numpy().astype(np.float64)
    bound = 2 * n * U32 * (np.abs(Ar.astype(np.float64)) @ np.abs(Bh.astype(np.float64)) + 0.5 * np.abs(Cr))
    slack = np.zeros_like(got)
    for x in rep.records:
        slack[rows.index(x["row"]), x["col"]] = x["tau"]
    assert np.all(np.abs(got - ref) <= bound + slack)
    _stat_check(got, ref, Ar, Bh, n, cin_abs=0.5 * np.abs(Cr))
    h.close()


def test_tc_bf16_16384_sampled_rows(ft, orc):
    import torch
    n = 16384
    Af = synth.torch_make("normal", (n, n), synth.workload_seed("tc_square", 0), "cuda")
    Bf = synth.torch_make("normal", (n, n), synth.workload_seed("tc_square", 1), "cuda")
    A, B = Af.to(torch.bfloat16), Bf.to(torch.bfloat16)
    del Af, Bf
    tm_n, tn_n, nks = -(-n // TDM_BF16), -(-n // TDN_BF16), n // 64
    pos = synth.fault_positions(synth.workload_seed("tc_square", 80), 16, tm_n, tn_n, nks, TDM_BF16, TDN_BF16, n, n, nks)
    faults = [(a, b, ks, r, c, float(64 * math.sqrt(n))) for (a, b, ks, r, c) in pos]
    h = ft.Handle(0)
    C = torch.empty(n, n, device="cuda")
    rep = h.gemm(A, B, C, level=ft.FT_TILE, dtype=ft.BF16, inject=faults)
    torch.cuda.synchronize()
    where = [(a * TDM_BF16 + r, b * TDN_BF16 + c) for (a, b, ks, r, c, d) in faults]
    assert sorted((x["row"], x["col"], x["kind"]) for x in rep.records) == sorted((i, j, 0) for i, j in where)
    rows = _rows(synth.workload_seed("tc_square", 81), n, [i for i, _ in where])
    Ar = A[rows].float().cpu().numpy()
    Bh = B.float().cpu().numpy()
    ref = orc.gemm_ref(Ar, Bh)
    got = C[rows].cpu().numpy().astype(np.float64)
    bound = 2 * n * U32 * (np.abs(Ar.astype(np.float64)) @ np.abs(Bh.astype(np.float64)))
    slack = np.zeros_like(got)
    for x in rep.records:
        slack[rows.index(x["row"]), x["col"]] = x["tau"]
    assert np.all(np.abs(got - ref) <= bound + slack)
    _stat_check(got, ref, Ar, Bh, n)
    h.close()


def test_group_512_sampled_problems(ft, orc):
    import torch
    nprob = 512
    u = synth.unit(synth.workload_seed("group512", 0), 3 * nprob)
    shapes = [(64 + 16 * int(u[3 * q] * 253), 64 + 16 * int(u[3 * q + 1] * 253), 64 + 16 * int(u[3 * q + 2] * 125))
              for q in range(nprob)]
    probs = []
    for q, (M, N, K) in enumerate(shapes):
        A = synth.torch_make("normal", (M, K), synth.workload_seed("group512", 100 + 2 * q), "cuda").to(torch.bfloat16)
        B = synth.torch_make("normal", (K, N), synth.workload_seed("group512", 101 + 2 * q), "cuda").to(torch.bfloat16)
        probs.append((A, B, torch.empty(M, N, device="cuda")))
    h = ft.Handle(0)
    g = ft.Group(h, probs, dtype=ft.BF16, level=ft.FT_TILE)
    tm, tn = g.tiles()
    tiles = sum(a * b for a, b in zip(tm, tn))
    nf = tiles // 100
    pick = synth.unit(synth.workload_seed("group512", 7), nf)
    by_prob = {}
    for f in range(nf):
        q = int(pick[f] * nprob)
        by_prob[q] = by_prob.get(q, 0) + 1
    faults = []
    for q, cnt in sorted(by_prob.items()):
        M, N, K = shapes[q]
        cnt = min(cnt, tm[q] * tn[q])
        for (a, b, ks, r, c) in synth.fault_positions(synth.workload_seed("group512", 1000 + q), cnt, tm[q], tn[q],
                                                      -(-K // 64), TDM_BF16, TDN_BF16, M, N, -(-K // 64)):
            faults.append((q, a, b, ks, r, c, float(64 * math.sqrt(K))))
    g.set_faults(faults)
    g.run()
    torch.cuda.synchronize()
    rep = h.report_fetch(capacity=1 << 15)
    want = sorted((f[0], f[1] * TDM_BF16 + f[4], f[2] * TDN_BF16 + f[5], 0) for f in faults)
    assert sorted((x["problem"], x["row"], x["col"], x["kind"]) for x in rep.records) == want
    # sampled problems in full, and every faulted problem among them
    sample = sorted(set(int(x * nprob) for x in synth.unit(synth.workload_seed("group512", 8), 6)) | {faults[0][0]})
    for q in sample:
        A, B, Cq = probs[q]
        Ah, Bh = A.float().cpu().numpy(), B.float().cpu().numpy()
        ref = orc.gemm_ref(Ah, Bh)
        got = Cq.cpu().numpy().astype(np.float64)
        K = Ah.shape[1]
        bound = 2 * K * U32 * (np.abs(Ah.astype(np.float64)) @ np.abs(Bh.astype(np.float64)))
        slack = np.zeros_like(got)
        for x in rep.records:
            if x["problem"] == q:
                slack[x["row"], x["col"]] = x["tau"]
        assert np.all(np.abs(got - ref) <= bound + slack)
        _stat_check(got, ref, Ah, Bh, K)
    g.close()
    h.close()


def test_tc_e4m3_16384_sampled_rows(ft, orc):
    """The tensor-core square in fp8: 16384^3 N(0,1) quantized to E4M3 with per-tensor
    scales, checksums through the MMA, 16 faults.  The quantizer matches the
    oracle's on sampled rows (the sample carries the tensor's largest
    element, so the per-tensor scale is the same); every fault is located
    and corrected; sampled rows of C match the oracle's product of the
    oracle-quantized operands."""
    import torch
    n = 16384
    tm_n, tn_n, nks = -(-n // TDM_E4M3), -(-n // TDN_E4M3), n // 128
    pos = synth.fault_positions(synth.workload_seed("tc_square", 23), 16, tm_n, tn_n, nks, TDM_E4M3, TDN_E4M3, n, n, nks)
    where = [(a * TDM_E4M3 + r, b * TDN_E4M3 + c) for (a, b, ks, r, c) in pos]
    rows = _rows(synth.workload_seed("tc_square", 22), n, [i for i, _ in where])
    Af = synth.torch_make("normal", (n, n), synth.workload_seed("tc_square", 20), "cuda")
    Bf = synth.torch_make("normal", (n, n), synth.workload_seed("tc_square", 21), "cuda")
    h = ft.Handle(0)
    A8, sa = h.quantize(Af, ft.E4M3)
    B8, sb = h.quantize(Bf, ft.E4M3)
    h.set_fp8_scales(sa, sb)
    # the oracle quantizes the sampled rows of A together with A's largest
    # element (so its per-tensor scale is A's), and all of B
    amax_idx = int(torch.argmax(Af.abs()).item())
    sample = np.concatenate([Af[rows].cpu().numpy().ravel(), Af.view(-1)[amax_idx:amax_idx + 1].cpu().numpy()])
    Bh = Bf.cpu().numpy()
    del Af, Bf
    _, q_s, sa_orc = orc.quant_e4m3(sample)
    _, Bq, sb_orc = orc.quant_e4m3(Bh)
    assert np.float32(sa) == np.float32(sa_orc) and np.float32(sb) == np.float32(sb_orc)
    Aq = q_s[:-1].reshape(len(rows), n)
    got_codes = A8[rows].cpu().view(torch.float8_e4m3fn).to(torch.float64).numpy()
    assert np.array_equal(got_codes, Aq)
    # offsets of 64 sqrt(K) in value units, i.e. / (sa sb) in units of the
    # accumulated code products
    faults = [(a, b, ks, r, c, float(64 * math.sqrt(n) / (sa * sb))) for (a, b, ks, r, c) in pos]
    C = torch.empty(n, n, device="cuda")
    rep = h.gemm(A8, B8, C, level=ft.FT_TILE, dtype=ft.E4M3, inject=faults)
    torch.cuda.synchronize()
    assert sorted((x["row"], x["col"], x["kind"]) for x in rep.records) == sorted((i, j, 0) for i, j in where)
    scale = np.float64(np.float32(sa)) * np.float64(np.float32(sb))
    ref = orc.gemm_ref(Aq, Bq) * scale
    got = C[rows].cpu().numpy().astype(np.float64)
    bound = (2 * n * U32 * (np.abs(Aq) @ np.abs(Bq))) * scale + 4 * U32 * np.abs(ref)
    slack = np.zeros_like(got)
    for x in rep.records:
        slack[rows.index(x["row"]), x["col"]] = x["tau"] * scale
    assert np.all(np.abs(got - ref) <= bound + slack)
    _stat_check(got, ref, Aq, Bq, n, scale=scale)
    h.close()
