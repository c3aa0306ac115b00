"""Bit-exact parity at the workloads' full sizes, on integer-valued inputs.

Integers uniform on [-4, 4] make every fp32 partial sum of these products
exact, in any order: at K = 16384 an element of C is at most 4*4*16384 = 2^18,
a tile checksum stays far below 2^24 (a random walk of about 10^4), and bf16
holds the operands exactly.  So the CUDA path must give the exact product,
whatever its tiling, raster, ring depth or wave count, and every injected
offset must come back as a residual equal to itself (the closed form of a
single fault, Eq. 3: d^r_i = d^c_j = delta, all other residuals 0).

Each case runs in the launch configuration bench.py times and checks
  * the record set equals the injected set, kind "corrected", with
    delta = residual_r = residual_c = the injected offset, verified at the end
    of the fault's period;
  * 16 or more sampled rows of C, every faulted row among them, equal the
    oracle's product exactly;
  * every row sum and every column sum of C equals A(Be) and (e^T A)B formed
    on the CPU in exact integer arithmetic (the ABFT identity of Eq. 3), so an
    element left wrong anywhere in C (a dropped k-slice, a missed tile of a
    late wave, an uncorrected fault) fails.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu
N_FULL = 16384
TDM_BF16, TDN = 125, 252  # bf16 tensor-core data tile with checksums (ftgemm_tc_tile)


@pytest.fixture(scope="module")
def ft():
    import torch
    import paper_2305_01024_gb300 as ft
    assert torch.cuda.is_available()
    ft.lib()
    return ft


def _offsets(seed, n, lo_exp=8, hi_exp=12):
    """Signed powers of two 2^lo_exp .. 2^hi_exp (exact in fp32 and bf16)."""
    u = synth.unit(seed, 2 * n)
    return [float((-1.0 if u[2 * q] < 0.5 else 1.0) * 2.0 ** (lo_exp + int(u[2 * q + 1] * (hi_exp - lo_exp + 1))))
            for q in range(n)]


def _int8_host(t):
    import torch
    return t.to(torch.int8).cpu().numpy()


def _line_sums_exact(A8, B8):
    """A(Be) and (e^T A)B in exact arithmetic on the CPU (float64 here holds
    every partial sum exactly: all values are integers far below 2^53)."""
    be = B8.sum(axis=1, dtype=np.int64).astype(np.float64)
    ea = A8.sum(axis=0, dtype=np.int64).astype(np.float64)
    rows = np.empty(A8.shape[0])
    for r0 in range(0, A8.shape[0], 2048):
        rows[r0:r0 + 2048] = A8[r0:r0 + 2048].astype(np.float64) @ be
    cols = np.zeros(B8.shape[1])
    for k0 in range(0, B8.shape[0], 2048):
        cols += ea[k0:k0 + 2048] @ B8[k0:k0 + 2048].astype(np.float64)
    return rows, cols


def _check_line_sums(C, A8, B8):
    import torch
    rows, cols = _line_sums_exact(A8, B8)
    Cd = C.double()
    got_r = Cd.sum(1).cpu().numpy()
    got_c = Cd.sum(0).cpu().numpy()
    assert np.array_equal(got_r, rows), f"{np.count_nonzero(got_r != rows)} row sums differ"
    assert np.array_equal(got_c, cols), f"{np.count_nonzero(got_c != cols)} column sums differ"
    del Cd
    torch.cuda.empty_cache()


def _check_records(rep, faults, tile_rows, tile_cols, period_end):
    want = sorted((tm * tile_rows + r, tn * tile_cols + c, 0, d, d, d, period_end(ks))
                  for (tm, tn, ks, r, c, d) in faults)
    got = sorted((x["row"], x["col"], x["kind"], x["delta"], x["residual_r"], x["residual_c"], x["kstep"])
                 for x in rep.records)
    assert got == want
    assert rep.corrected == len(faults) and rep.uncorrectable == 0 and rep.checksum_only == 0


def _check_rows(orc, C, A_host, B_host, rows):
    ref = orc.gemm_ref(A_host[rows], B_host)
    got = C[rows].double().cpu().numpy()
    assert np.array_equal(got, ref), f"{np.count_nonzero(got != ref)} sampled elements differ"


def _sample_rows(seed, M, faulted):
    return sorted(set(int(u * M) for u in synth.unit(seed, 12)) | set(faulted))


def test_headline_fp32_block_16384_integers_bit_exact(ft, orc):
    """The headline schedule (128 x 128 tile, 64 x 64 warps, 16 x 8 fragments,
    k-steps of 32 in a 3-deep ring, block-level checksums verified every 8
    k-steps) over 16384^3 integers: 128 x 128 tiles in the grouped raster,
    several waves of two CTAs per SM."""
    import torch
    n = N_FULL
    sched = dict(m_tb=128, n_tb=128, k_tb=32, m_w=64, n_w=64, m_t=16, n_t=8, cadence=8, split_k=1)
    A = synth.torch_make("int", (n, n), synth.workload_seed("sweep_fp32", 40), "cuda")
    B = synth.torch_make("int", (n, n), synth.workload_seed("sweep_fp32", 41), "cuda")
    tiles, ksteps = n // 128, n // 32
    pos = synth.fault_positions(synth.workload_seed("sweep_fp32", 42), 16, tiles, tiles, ksteps, 128, 128, n, n, 8)
    faults = [p + (d,) for p, d in zip(pos, _offsets(synth.workload_seed("sweep_fp32", 43), 16))]
    h = ft.Handle(0)
    h.set_schedule(sched)
    C = torch.full((n, n), float("nan"), device="cuda")
    rep = h.gemm(A, B, C, alpha=1.0, beta=0.0, level=ft.FT_BLOCK, inject=faults)
    torch.cuda.synchronize()
    _check_records(rep, faults, 128, 128, lambda ks: (ks // 8) * 8 + 7)
    A8, B8 = _int8_host(A), _int8_host(B)
    rows = _sample_rows(synth.workload_seed("sweep_fp32", 44), n, [f[0] * 128 + f[3] for f in faults])
    assert len(rows) >= 16
    _check_rows(orc, C, A8.astype(np.float32), B8.astype(np.float32), rows)
    _check_line_sums(C, A8, B8)
    h.close()


def test_tile_bf16_16384_integers_bit_exact(ft, orc):
    """bf16 TILE at 16384^3 (the persistent tcgen05 kernel over 132 x 66 tiles
    of 125 x 252, checksums carried through the MMA), integer operands."""
    import torch
    n = N_FULL
    A = synth.torch_make("int", (n, n), synth.workload_seed("tc_square", 40), "cuda").to(torch.bfloat16)
    B = synth.torch_make("int", (n, n), synth.workload_seed("tc_square", 41), "cuda").to(torch.bfloat16)
    tm_n, tn_n, nks = -(-n // TDM_BF16), -(-n // TDN), n // 64
    pos = synth.fault_positions(synth.workload_seed("tc_square", 42), 16, tm_n, tn_n, nks, TDM_BF16, TDN, n, n, nks)
    faults = [p + (d,) for p, d in zip(pos, _offsets(synth.workload_seed("tc_square", 43), 16))]
    h = ft.Handle(0)
    C = torch.full((n, n), float("nan"), device="cuda")
    rep = h.gemm(A, B, C, level=ft.FT_TILE, dtype=ft.BF16, inject=faults)
    torch.cuda.synchronize()
    _check_records(rep, faults, TDM_BF16, TDN, lambda ks: nks - 1)
    A8, B8 = _int8_host(A), _int8_host(B)
    rows = _sample_rows(synth.workload_seed("tc_square", 44), n, [f[0] * TDM_BF16 + f[3] for f in faults])
    assert len(rows) >= 16
    _check_rows(orc, C, A8.astype(np.float32), B8.astype(np.float32), rows)
    _check_line_sums(C, A8, B8)
    h.close()


def test_group_512_bf16_integers_bit_exact(ft, orc):
    """The grouped workload's 512 problems (M, N on 64..4096, K on 64..2048, steps of 16)
    in one persistent grouped launch, integer operands in bf16, 1% of the
    tiles faulted: every problem's row and column sums exact, the record set
    exact, sampled problems (every faulted one of the first few among them)
    exact element by element."""
    import torch
    nprob = 512
    u = synth.unit(synth.workload_seed("group512", 0), 3 * nprob)
    shapes = [(64 + 16 * int(u[3 * q] * 253), 64 + 16 * int(u[3 * q + 1] * 253), 64 + 16 * int(u[3 * q + 2] * 125))
              for q in range(nprob)]
    probs = []
    for q, (M, N, K) in enumerate(shapes):
        A = synth.torch_make("int", (M, K), synth.workload_seed("group512", 300 + 2 * q), "cuda").to(torch.bfloat16)
        B = synth.torch_make("int", (K, N), synth.workload_seed("group512", 301 + 2 * q), "cuda").to(torch.bfloat16)
        probs.append((A, B, torch.full((M, N), float("nan"), device="cuda")))
    h = ft.Handle(0)
    g = ft.Group(h, probs, dtype=ft.BF16, level=ft.FT_TILE)
    tm, tn = g.tiles()
    tiles = sum(a * b for a, b in zip(tm, tn))
    nf = tiles // 100
    pick = synth.unit(synth.workload_seed("group512", 47), nf)
    by_prob = {}
    for f in range(nf):
        q = int(pick[f] * nprob)
        by_prob[q] = by_prob.get(q, 0) + 1
    faults = []
    for q, cnt in sorted(by_prob.items()):
        M, N, K = shapes[q]
        cnt = min(cnt, tm[q] * tn[q])
        nkb = -(-K // 64)
        sites = synth.fault_positions(synth.workload_seed("group512", 2000 + q), cnt, tm[q], tn[q], nkb, TDM_BF16, TDN, M, N, nkb)
        for (a, b, ks, r, c), d in zip(sites, _offsets(synth.workload_seed("group512", 3000 + q), cnt)):
            faults.append((q, a, b, ks, r, c, d))
    g.set_faults(faults)
    g.run()
    torch.cuda.synchronize()
    rep = h.report_fetch(capacity=1 << 15)
    want = sorted((f[0], f[1] * TDM_BF16 + f[4], f[2] * TDN + f[5], 0, f[6], f[6], f[6]) for f in faults)
    got = sorted((x["problem"], x["row"], x["col"], x["kind"], x["delta"], x["residual_r"], x["residual_c"])
                 for x in rep.records)
    assert got == want
    for q, (A, B, Cq) in enumerate(probs):
        _check_line_sums(Cq, _int8_host(A), _int8_host(B))
    faulted = sorted({f[0] for f in faults})
    sample = sorted(set(int(x * nprob) for x in synth.unit(synth.workload_seed("group512", 48), 4)) | set(faulted[:4]))
    for q in sample:
        A, B, Cq = probs[q]
        Ah, Bh = _int8_host(A).astype(np.float32), _int8_host(B).astype(np.float32)
        ref = orc.gemm_ref(Ah, Bh)
        assert np.array_equal(Cq.double().cpu().numpy(), ref), f"problem {q} differs"
    g.close()
    h.close()
