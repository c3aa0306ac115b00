"""Pins for the CPU oracle (no GPU).

Every check here compares the oracle with something other than itself: a
hand-worked fixture, plain-Python brute force on tiny inputs, closed forms of
the single-fault residual, numpy/torch library routines, or a Monte-Carlo
simulation.  Each is chosen so that a plausible slip in the oracle (a dropped
term, a wrong sign or index, a transposed operand, a wrong unit layout) fails.
"""
import itertools
import os

import numpy as np
import pytest

import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden", "eq1_3_worked_example.txt")


def _parse_golden():
    exs, cur = [], None
    for line in open(GOLD):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        if line.startswith("A "):
            cur = {}
            exs.append(cur)
        key, _, vals = line.partition(":")
        key = key.split()
        if key[0] == "fault":
            kv = dict(x.split("=") for x in key[1:])
            cur["fault"] = (int(kv["row"]), int(kv["col"]), float(kv["delta"]))
            continue
        nums = [float(x) for x in vals.split()]
        if key[0] in ("A", "B"):
            cur[key[0]] = np.array(nums).reshape(int(key[1]), int(key[2]))
        else:
            cur[key[0]] = np.array(nums)
    return exs


def _sched(orc, M, N, K, level=None, **kw):
    level = orc.BLOCK if level is None else level
    return orc.Schedule(m_tb=M, n_tb=N, k_tb=K, m_w=M, n_w=N, m_t=M, n_t=N,
                        cadence=1, level=level, **kw)


# --------------------------------------------------------------------------
# Eq. 1-3 worked examples
# --------------------------------------------------------------------------

@pytest.mark.parametrize("ex", range(2))
def test_golden_encoding_and_product(orc, ex):
    g = _parse_golden()[ex]
    A, B = g["A"], g["B"]
    M, K = A.shape
    N = B.shape[1]
    V, W, nA, nB = orc.encode(A, B, m_u=M, n_u=N)
    assert np.array_equal(V[0], g["eTA"])
    assert np.array_equal(W[0], g["Be"])
    C = orc.gemm_ref(A, B)
    assert np.array_equal(C.ravel(), g["C"])
    assert np.array_equal(C.sum(axis=1), g["Ce"])
    assert np.array_equal(C.sum(axis=0), g["eTC"])


@pytest.mark.parametrize("ex", range(2))
def test_golden_single_fault_residuals(orc, ex):
    g = _parse_golden()[ex]
    A, B = g["A"], g["B"]
    M, K = A.shape
    N = B.shape[1]
    r, c, delta = g["fault"]
    res = orc.gemm_ft(A, B, _sched(orc, M, N, K), faults=[(0, 0, 0, r, c, delta)])
    assert (res.detected, res.corrected) == (1, 1)
    rec = res.records[0]
    assert (rec.row, rec.col) == (r, c)
    # the only non-zero residuals are the fixture's
    assert rec.residual_r == g["dr"][r] and rec.residual_c == g["dc"][c]
    assert rec.delta == delta
    assert np.array_equal(res.C.ravel(), g["C"])


# --------------------------------------------------------------------------
# Plain definition and the fault-free ABFT path vs brute force
# --------------------------------------------------------------------------

def _brute(A, B, alpha, beta, Cin):
    M, K = A.shape
    N = B.shape[1]
    out = [[0.0] * N for _ in range(M)]
    for i in range(M):
        for j in range(N):
            s = 0.0
            for k in range(K):
                s += float(A[i, k]) * float(B[k, j])
            out[i][j] = alpha * s + (beta * float(Cin[i, j]) if beta else 0.0)
    return np.array(out)


@pytest.mark.parametrize("M,N,K", [(1, 1, 1), (1, 9, 2), (9, 1, 3), (3, 5, 7), (7, 4, 9), (9, 9, 9)])
def test_brute_force_tiny_integer(orc, M, N, K):
    A = synth.integers((M, K), 11 + M)
    B = synth.integers((K, N), 12 + N)
    Cin = synth.integers((M, N), 13 + K)
    ref = _brute(A, B, 2.0, -3.0, Cin)
    assert np.array_equal(orc.gemm_ref(A, B, 2.0, -3.0, Cin), ref)
    for level in (orc.THREAD, orc.WARP, orc.BLOCK):
        s = orc.Schedule(m_tb=4, n_tb=4, k_tb=2, m_w=2, n_w=4, m_t=1, n_t=1,
                         cadence=2, level=level)
        # thread fragment 1x1 (lanes 2x4) is a legal unit layout for the tiny case
        res = orc.gemm_ft(A, B, s, alpha=2.0, beta=-3.0, Cin=Cin)
        assert np.array_equal(res.C, ref), level
        assert res.detected == 0


def test_float_matches_numpy_float64(orc):
    A = synth.uniform((67, 45), 1)
    B = synth.uniform((45, 53), 2)
    Cin = synth.uniform((67, 53), 3)
    ref = 0.75 * (A.astype(np.float64) @ B.astype(np.float64)) + 0.5 * Cin
    out = orc.gemm_ref(A, B, 0.75, 0.5, Cin)
    assert np.max(np.abs(out - ref)) <= 1e-13
    res = orc.gemm_ft(A, B, orc.Schedule(m_tb=32, n_tb=32, k_tb=8, m_w=16, n_w=32,
                                         m_t=4, n_t=4, cadence=2), alpha=0.75, beta=0.5, Cin=Cin)
    assert np.max(np.abs(res.C - ref)) <= 1e-13
    assert res.detected == 0


def test_identity_eTAB_equals_eTA_B_exact(orc):
    """e^T(AB) = (e^T A)B and (AB)e = A(Be) per block, exactly on integers (Eq. 3)."""
    M, N, K, mu, nu = 70, 50, 33, 16, 8
    A = synth.integers((M, K), 5)
    B = synth.integers((K, N), 6)
    V, W, nA, nB = orc.encode(A, B, mu, nu)
    Ai, Bi = A.astype(np.int64), B.astype(np.int64)
    C = Ai @ Bi  # exact integer product (numpy)
    for b in range(V.shape[0]):
        rows = slice(b * mu, min(M, (b + 1) * mu))
        assert np.array_equal(V[b].astype(np.int64) @ Bi, C[rows].sum(axis=0))
    for b in range(W.shape[0]):
        cols = slice(b * nu, min(N, (b + 1) * nu))
        assert np.array_equal(Ai @ W[b].astype(np.int64), C[:, cols].sum(axis=1))
    assert np.allclose(nA, np.linalg.norm(A.astype(np.float64), axis=1), rtol=1e-14)
    assert np.allclose(nB, np.linalg.norm(B.astype(np.float64), axis=0), rtol=1e-14)


# --------------------------------------------------------------------------
# Fault handling, closed forms
# --------------------------------------------------------------------------

HUGE = dict(m_tb=128, n_tb=128, k_tb=8, m_w=32, n_w=64, m_t=8, n_t=8)


def _thread_unit(r, c, m_w=32, n_w=64, m_t=8, n_t=8):
    """Independent restatement of the 4x8-lane fragment ownership (Table 1 layout)."""
    lm, ln = m_w // m_t, n_w // n_t
    vm, vn = min(4, m_t), min(4, n_t)
    tm = (r % m_w) % (lm * vm) // vm
    tn = (c % n_w) % (ln * vn) // vn
    return (r // m_w, tm, c // n_w, tn)


@pytest.mark.parametrize("level", ["BLOCK", "WARP", "THREAD"])
def test_int256_style_faults_corrected_bitwise(orc, level):
    """256^3 integers, 4 faults of +2^10 at distinct units/periods: all corrected, C exact."""
    M = N = K = 256
    A = synth.integers((M, K), synth.workload_seed("int256", 0))
    B = synth.integers((K, N), synth.workload_seed("int256", 1))
    lv = getattr(orc, level)
    s = orc.Schedule(**HUGE, cadence=4, level=lv)
    unit_of = {"BLOCK": lambda r, c: 0, "WARP": lambda r, c: (r // 32, c // 64),
               "THREAD": _thread_unit}[level]
    pos = synth.fault_positions(synth.workload_seed("int256", 2), 4, 2, 2, 32, 128, 128, M, N, 4,
                                unit_of=unit_of)
    faults = [p + (1024.0,) for p in pos]
    clean = orc.gemm_ft(A, B, s)
    res = orc.gemm_ft(A, B, s, faults=faults)
    ref = A.astype(np.int64) @ B.astype(np.int64)
    assert np.array_equal(clean.C, ref)
    assert np.array_equal(res.C, ref)
    assert (res.detected, res.corrected, res.uncorrectable, res.checksum_only) == (4, 4, 0, 0)
    got = sorted((r.tile_m, r.tile_n, r.row, r.col) for r in res.records)
    want = sorted((tm, tn, tm * 128 + r, tn * 128 + c) for tm, tn, ks, r, c in pos)
    assert got == want
    for r in res.records:
        assert r.delta == 1024.0 and r.residual_r == 1024.0 and r.residual_c == 1024.0
        # verified at the end of the fault's period (cadence 4 k-steps)
        f = [p for p in pos if (p[0], p[1]) == (r.tile_m, r.tile_n)
             and p[0] * 128 + p[3] == r.row][0]
        assert r.kstep == (f[2] // 4) * 4 + 3


def test_two_faults_same_unit_same_period_uncorrectable(orc):
    """Single-event-upset model (Section 4.1): two faults in one period are not correctable."""
    M = N = K = 128
    A = synth.integers((M, K), 21)
    B = synth.integers((K, N), 22)
    s = orc.Schedule(**HUGE, cadence=4, level=orc.BLOCK)
    res = orc.gemm_ft(A, B, s, faults=[(0, 0, 1, 3, 5, 64.0), (0, 0, 2, 9, 70, 32.0)])
    ref = A.astype(np.int64) @ B.astype(np.int64)
    # reported at its period (k-steps 0..3) and again at each of the 3 later ones,
    # because an uncorrectable unit stays corrupted
    assert (res.detected, res.corrected, res.uncorrectable) == (4, 0, 4)
    assert [r.kstep for r in res.records] == [3, 7, 11, 15]
    diff = res.C - ref
    assert diff[3, 5] == 64.0 and diff[9, 70] == 32.0 and np.count_nonzero(diff) == 2


def test_two_faults_same_unit_different_periods_corrected(orc):
    M = N = K = 128
    A = synth.integers((M, K), 21)
    B = synth.integers((K, N), 22)
    s = orc.Schedule(**HUGE, cadence=4, level=orc.BLOCK)
    res = orc.gemm_ft(A, B, s, faults=[(0, 0, 1, 3, 5, 64.0), (0, 0, 6, 3, 5, -32.0)])
    assert (res.detected, res.corrected) == (2, 2)
    assert np.array_equal(res.C, A.astype(np.int64) @ B.astype(np.int64))
    assert [r.kstep for r in res.records] == [3, 7]


def test_thread_units_separate_faults_one_block_period(orc):
    """Same tile and period, different thread fragments: the THREAD level corrects
    both, the BLOCK level cannot (pins the fragment layout of the unit)."""
    M = N = K = 128
    A = synth.integers((M, K), 31)
    B = synth.integers((K, N), 32)
    # (0,0) and (4,4): thread (tm=0,tn=0) vs (tm=1,tn=1); (16,32) shares thread (0,0)
    f_sep = [(0, 0, 0, 0, 0, 8.0), (0, 0, 0, 4, 4, 8.0)]
    f_same = [(0, 0, 0, 0, 0, 8.0), (0, 0, 0, 16, 32, 8.0)]
    ref = A.astype(np.int64) @ B.astype(np.int64)
    for faults, lvl, ok in [(f_sep, orc.THREAD, True), (f_sep, orc.BLOCK, False),
                            (f_same, orc.THREAD, False), (f_same, orc.WARP, False)]:
        res = orc.gemm_ft(A, B, orc.Schedule(**HUGE, cadence=16, level=lvl), faults=faults)
        assert np.array_equal(res.C, ref) == ok, (faults, lvl)
        assert _thread_unit(0, 0) != _thread_unit(4, 4)
        assert _thread_unit(0, 0) == _thread_unit(16, 32)


WIDE32 = dict(m_tb=128, n_tb=128, k_tb=32, m_w=64, n_w=64, m_t=16, n_t=8)


def test_thread_units_of_the_16x8_fragment(orc):
    """The headline tuple's thread fragments (64 x 64 warp tile, 4 x 8 lanes,
    16 x 8 per lane): a lane's 16 rows come as 4 chunks of 4 consecutive rows,
    16 apart, and its 8 columns as 2 chunks of 4, 32 apart.  Rows 0 and 8
    belong to different lanes (a contiguous 16-row fragment would merge them),
    rows 0 and 16 to the same lane (chunk 0 and 1 of lane row 0), columns 0
    and 32 to the same lane, columns 0 and 16 to different ones; rows 0 and 64
    lie in different warp tiles.  Two faults in one period are both corrected
    at the THREAD level exactly when they fall in different fragments."""
    M = N = K = 128
    A = synth.integers((M, K), 33)
    B = synth.integers((K, N), 34)
    ref = A.astype(np.int64) @ B.astype(np.int64)
    unit = lambda r, c: _thread_unit(r, c, m_w=64, n_w=64, m_t=16, n_t=8)
    cases = [((0, 0), (8, 0), True), ((0, 0), (16, 0), False), ((0, 0), (0, 32), False),
             ((0, 0), (0, 16), True), ((3, 3), (51, 35), False), ((0, 0), (64, 0), True),
             ((0, 0), (4, 4), True)]
    for (r0, c0), (r1, c1), sep in cases:
        assert (unit(r0, c0) != unit(r1, c1)) == sep, ((r0, c0), (r1, c1))
        faults = [(0, 0, 1, r0, c0, 8.0), (0, 0, 1, r1, c1, -16.0)]
        res = orc.gemm_ft(A, B, orc.Schedule(**WIDE32, cadence=2, level=orc.THREAD), faults=faults)
        assert np.array_equal(res.C, ref) == sep, ((r0, c0), (r1, c1))
        if sep:
            assert res.corrected == 2 and res.uncorrectable == 0
        else:
            assert res.uncorrectable >= 1


def test_warp_units_follow_the_warp_tile(orc):
    """Same tile and period (Section 4.2.2): faults in different m_w x n_w warp
    tiles are both corrected at the WARP level, while the BLOCK level sees two
    flagged rows or columns; two faults inside one warp tile defeat WARP too.
    The tuple's warp tile is 32 x 64."""
    M = N = K = 128
    A = synth.integers((M, K), 41)
    B = synth.integers((K, N), 42)
    ref = A.astype(np.int64) @ B.astype(np.int64)
    below = [(0, 0, 2, 0, 0, 16.0), (0, 0, 2, 32, 0, 16.0)]    # warp rows 0 and 1, column 0
    beside = [(0, 0, 2, 5, 3, 16.0), (0, 0, 2, 5, 64, -16.0)]  # warp columns 0 and 1, row 5
    inside = [(0, 0, 2, 0, 0, 16.0), (0, 0, 2, 31, 63, 16.0)]  # both in warp tile (0, 0)
    for faults, lvl, ok in [(below, orc.WARP, True), (below, orc.BLOCK, False),
                            (beside, orc.WARP, True), (beside, orc.BLOCK, False),
                            (inside, orc.WARP, False)]:
        res = orc.gemm_ft(A, B, orc.Schedule(**HUGE, cadence=16, level=lvl), faults=faults)
        assert np.array_equal(res.C, ref) == ok, (faults, lvl)
        if ok:
            assert res.corrected == 2 and res.uncorrectable == 0
            assert sorted((r.row, r.col) for r in res.records) == sorted((f[3], f[4]) for f in faults)
        else:
            assert res.uncorrectable >= 1


@pytest.mark.parametrize("target,kind_row", [(1, True), (2, False)])
def test_checksum_hit_is_reported_and_c_untouched(orc, target, kind_row):
    M = N = K = 64
    A = synth.integers((M, K), 41)
    B = synth.integers((K, N), 42)
    s = orc.Schedule(m_tb=64, n_tb=64, k_tb=8, m_w=32, n_w=32, m_t=4, n_t=4,
                     cadence=2, level=orc.BLOCK)
    res = orc.gemm_ft(A, B, s, faults=[(0, 0, 2, 7, 9, 100.0, target)])
    assert (res.detected, res.checksum_only, res.corrected) == (1, 1, 0)
    rec = res.records[0]
    assert rec.kind == orc.CHECKSUM_ONLY and rec.delta == 100.0
    assert (rec.row == 7) == kind_row and (rec.col == 9) == (not kind_row)
    assert np.array_equal(res.C, A.astype(np.int64) @ B.astype(np.int64))


def test_ragged_tiles_split_k_alpha_beta(orc):
    M, N, K = 77, 45, 70
    A = synth.integers((M, K), 51)
    B = synth.integers((K, N), 52)
    Cin = synth.integers((M, N), 53)
    s = orc.Schedule(m_tb=32, n_tb=32, k_tb=4, m_w=16, n_w=32, m_t=4, n_t=4,
                     cadence=3, split_k=3, level=orc.BLOCK)
    # last ragged tile (2, 1): 13 rows x 13 cols; k-step -1 = the last one
    faults = [(2, 1, -1, 12, 12, 512.0), (0, 0, 9, 0, 31, -256.0)]
    res = orc.gemm_ft(A, B, s, faults=faults, alpha=-1.0, beta=2.0, Cin=Cin)
    ref = -(A.astype(np.int64) @ B.astype(np.int64)) + 2 * Cin.astype(np.int64)
    assert np.array_equal(res.C, ref)
    assert res.corrected == 2
    ks = {(r.tile_m, r.tile_n): r.kstep for r in res.records}
    assert ks[(2, 1)] == 17  # 18 k-steps in total, -1 -> 17
    assert ks[(0, 0)] == 11  # split 2 owns k-steps 6..11; local period ends at 8 and 11


def test_out_of_range_fault_is_ignored(orc):
    A = synth.integers((40, 16), 61)
    B = synth.integers((16, 40), 62)
    s = orc.Schedule(m_tb=32, n_tb=32, k_tb=8, m_w=16, n_w=32, m_t=4, n_t=4, cadence=1)
    res = orc.gemm_ft(A, B, s, faults=[(1, 1, 0, 20, 3, 9.0)])  # tile (1,1) has 8 rows
    assert res.detected == 0


def test_float_no_false_alarm_and_fault_found(orc):
    """U(-1,1) fp32 inputs: no flags without faults; a fault 1e-2 x the tile's
    max |C| is flagged, located and corrected."""
    M = N = 256
    K = 512
    A = synth.uniform((M, K), 71)
    B = synth.uniform((K, N), 72)
    s = orc.Schedule(**HUGE, cadence=16)
    clean = orc.gemm_ft(A, B, s)
    assert clean.detected == 0
    tmax = np.abs(clean.C[:128, :128]).max()
    res = orc.gemm_ft(A, B, s, faults=[(0, 0, 20, 5, 6, 1e-2 * tmax)])
    assert res.corrected == 1 and res.records[0].row == 5 and res.records[0].col == 6
    assert np.max(np.abs(res.C - clean.C)) < 1e-9


# --------------------------------------------------------------------------
# Low-precision conversions vs library routines
# --------------------------------------------------------------------------

def test_bf16_rounding_matches_torch(orc):
    torch = pytest.importorskip("torch")
    x = np.concatenate([synth.normal((4096,), 81) * 10.0 ** synth.integers((4096,), 82, -30, 30),
                        np.array([0.0, -0.0, 1.0, 1.00390625, 1.01171875, 3.3e38, 1e-40],
                                 dtype=np.float32)]).astype(np.float32)
    ours = orc.round_bf16(x)
    theirs = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(ours, theirs)


def test_e4m3_quantization_matches_torch(orc):
    torch = pytest.importorskip("torch")
    if not hasattr(torch, "float8_e4m3fn"):
        pytest.skip("torch without float8")
    x = synth.normal((8192,), 91)
    deq, q, scale = orc.quant_e4m3(x)
    assert scale == np.float32(np.abs(x).max()) / np.float32(448.0)
    xs = torch.from_numpy(x) / torch.tensor(scale, dtype=torch.float32)
    theirs = xs.to(torch.float8_e4m3fn).to(torch.float64).numpy()
    assert np.array_equal(q, theirs)
    assert np.abs(q).max() == 448.0


def test_bf16_hand_worked_values(orc):
    # bf16: 8 exponent bits (as fp32), 7 stored mantissa bits, round to
    # nearest with ties to the even mantissa.  Spacing is 2^-7 on [1, 2),
    # 2 on [256, 512) and 2^-133 among the subnormals.
    cases = [
        (1.0 + 2.0 ** -8, 1.0),                      # tie: mantissa 0 (even) wins
        (1.0 + 3 * 2.0 ** -8, 1.0 + 2.0 ** -6),      # tie between 1 (odd) and 2 (even)
        (1.0 + 2.0 ** -8 + 2.0 ** -16, 1.0 + 2.0 ** -7),  # just above the tie
        (256.5, 256.0),
        (257.0, 256.0),                              # tie between 256 and 258
        (259.0, 260.0),                              # tie between 258 and 260
        (-3.0, -3.0),
        (2.0 ** -130, 2.0 ** -130),                  # subnormal, representable
        (1.5 * 2.0 ** -133, 2.0 ** -132),            # subnormal tie to even
        ((2.0 - 2.0 ** -7) * 2.0 ** 127, (2.0 - 2.0 ** -7) * 2.0 ** 127),  # largest finite
        (0.0, 0.0),
    ]
    x = np.array([c[0] for c in cases], dtype=np.float32)
    assert np.array_equal(x.astype(np.float64), [c[0] for c in cases])  # inputs exact in fp32
    assert list(orc.round_bf16(x)) == [c[1] for c in cases]
    # 0.1f = 1.6000000238 * 2^-4: 204.80000305 / 128 rounds to 205 / 128
    assert orc.round_bf16(np.array([0.1], np.float32))[0] == 205 / 128 * 2.0 ** -4


def test_e4m3_hand_worked_values(orc):
    # OCP FP8 E4M3: bias 7, 3 mantissa bits, largest finite 1.75 * 2^8 = 448,
    # smallest normal 2^-6, subnormal spacing 2^-9; round to nearest even,
    # saturating.  448 is in the input, so the per-tensor scale
    # amax / 448 is exactly 1 and q holds the codes' values directly.
    cases = [
        (448.0, 448.0),
        (1.0625, 1.0),                  # tie between 1.0 (even) and 1.125
        (1.1875, 1.25),                 # tie between 1.125 (odd) and 1.25
        (17.0, 16.0),                   # spacing 2 on [16, 32): tie to 16
        (19.0, 20.0),
        (240.0, 240.0),                 # 1.875 * 2^7, exact
        (248.0, 256.0),                 # tie between 240 (odd) and 256 (even)
        (440.0, 448.0),                 # above the 432 midpoint
        (0.3, 0.3125),                  # spacing 2^-5 on [0.25, 0.5): 9.6 -> 10
        (2.0 ** -9, 2.0 ** -9),         # smallest subnormal
        (2.0 ** -10, 0.0),              # tie between 0 (even) and 2^-9
        (3 * 2.0 ** -10, 2.0 ** -8),    # tie between 1 and 2 subnormal steps
        (7 * 2.0 ** -9, 7 * 2.0 ** -9),  # largest subnormal
        (7.5 * 2.0 ** -9, 2.0 ** -6),   # tie into the smallest normal
        (-1.0625, -1.0),
        (0.0, 0.0),
    ]
    x = np.array([c[0] for c in cases], dtype=np.float32)
    deq, q, scale = orc.quant_e4m3(x)
    assert scale == 1.0
    assert list(q) == [c[1] for c in cases]
    assert np.array_equal(deq, q)
    # a scale of 2: amax 896 maps to 448, and the codes are those of x / 2
    # (-150: spacing 16 on [128, 256), 9.375 -> 9; 50: spacing 4, 12.5 -> 12)
    y = np.array([896.0, -300.0, 100.0], np.float32)
    _, qy, sy = orc.quant_e4m3(y)
    assert sy == 2.0 and list(qy) == [448.0, -144.0, 48.0]


# --------------------------------------------------------------------------
# Section 5.5 cost model vs a Monte-Carlo simulation of the restart process
# --------------------------------------------------------------------------

def test_offline_expected_runs_monte_carlo(orc):
    rng = np.random.default_rng(7)
    gamma0, tiles = 1 / 256, 40
    gamma = 1 - (1 - gamma0) ** tiles
    # each run fails with prob gamma; a failure costs the run plus two more tries'
    # worth of exposure as the paper's recursion (1-g) + 2g((1-g) + 2g(...)) states
    trials = 200_000
    runs = np.ones(trials)
    weight = np.ones(trials)
    alive = np.ones(trials, dtype=bool)
    total = np.zeros(trials)
    for _ in range(60):
        fail = rng.random(trials) < gamma
        total += np.where(alive & ~fail, weight, 0.0)
        weight = np.where(alive & fail, weight * 2, weight)
        alive &= fail
        if not alive.any():
            break
    est = total.mean()
    assert abs(est - orc.offline_expected_runs(gamma0, tiles)) < 0.01
    assert orc.offline_expected_runs(gamma0, tiles) > 1.0
    assert orc.offline_expected_runs(0.3, 4) == float("inf")


def test_offline_expected_runs_closed_forms(orc):
    # gamma = 1 - (1 - gamma0)^tiles, runs = (1 - gamma) / (1 - 2 gamma), by hand:
    assert orc.offline_expected_runs(0.0, 64) == 1.0              # no errors: one run
    assert abs(orc.offline_expected_runs(0.25, 1) - 1.5) < 1e-15  # (3/4) / (1/2)
    assert abs(orc.offline_expected_runs(1 / 256, 1) - 255 / 254) < 1e-15
    # two tiles at 1/2: gamma = 3/4 >= 1/2, the restart series diverges
    assert orc.offline_expected_runs(0.5, 2) == float("inf")
    # more tiles, more exposure: the expectation grows with the tile count
    r = [orc.offline_expected_runs(1 / 256, t) for t in (16, 64, 144)]
    assert 1.0 < r[0] < r[1] < r[2]


# --------------------------------------------------------------------------
# Detect-only (the offline scheme of Section 5.5)
# --------------------------------------------------------------------------

DET = dict(m_tb=128, n_tb=128, k_tb=32, m_w=64, n_w=64, m_t=16, n_t=8)


def test_detect_only_reports_the_column_and_corrects_nothing(orc):
    """Integer inputs, one offset per tile: each tile reports one detection
    at the split's end, at the faulted column with residual exactly the
    offset, no row; C keeps every offset (the offline scheme recomputes)."""
    M, N, K = 256, 256, 512
    A = synth.integers((M, K), 81)
    B = synth.integers((K, N), 82)
    ref = A.astype(np.int64) @ B.astype(np.int64)
    faults = [(0, 0, 3, 5, 9, 64.0), (1, 1, 10, 100, 17, -32.0), (0, 1, 15, 0, 127, 8.0)]
    s = orc.Schedule(**DET, cadence=K // 32, level=orc.DETECT)
    res = orc.gemm_ft(A, B, s, faults=faults)
    assert (res.detected, res.corrected, res.uncorrectable, res.checksum_only) == (3, 0, 3, 0)
    got = sorted((r.tile_m, r.tile_n, r.kstep, r.row, r.col, r.kind, r.residual_c) for r in res.records)
    want = sorted((tm, tn, K // 32 - 1, -1, tn * 128 + c, orc.UNCORRECTABLE, d) for (tm, tn, ks, r, c, d) in faults)
    assert got == want
    diff = res.C - ref
    assert np.count_nonzero(diff) == 3
    for (tm, tn, ks, r, c, d) in faults:
        assert diff[tm * 128 + r, tn * 128 + c] == d


def test_detect_only_checks_columns_only(orc):
    """A hit on a row checksum goes unseen (the detector keeps none); a hit
    on a column checksum is a detection; two offsets in one tile give one
    record, at the column with the larger |residual| / tau."""
    M, N, K = 128, 128, 256
    A = synth.integers((M, K), 83)
    B = synth.integers((K, N), 84)
    s = orc.Schedule(**DET, cadence=K // 32, level=orc.DETECT)
    row_hit = orc.gemm_ft(A, B, s, faults=[(0, 0, 2, 5, 9, 64.0, orc.T_ROWSUM)])
    assert row_hit.detected == 0
    col_hit = orc.gemm_ft(A, B, s, faults=[(0, 0, 2, 5, 9, 64.0, orc.T_COLSUM)])
    assert col_hit.detected == 1 and col_hit.records[0].col == 9 and col_hit.records[0].residual_c == -64.0
    two = orc.gemm_ft(A, B, s, faults=[(0, 0, 2, 5, 9, 64.0), (0, 0, 3, 70, 40, -128.0)])
    assert two.detected == 1 and two.records[0].col == 40


def test_detect_only_split_k_and_float_inputs(orc):
    """With split-K each split reports at its own end; fault-free float
    inputs raise nothing."""
    M, N, K = 128, 256, 1024
    A = synth.integers((M, K), 85)
    B = synth.integers((K, N), 86)
    s = orc.Schedule(**DET, cadence=K // 64, split_k=2, level=orc.DETECT)
    res = orc.gemm_ft(A, B, s, faults=[(0, 1, 3, 1, 2, 16.0), (0, 0, 20, 7, 8, 16.0)])
    assert sorted((r.tile_n, r.kstep) for r in res.records) == [(0, 31), (1, 15)]
    Af = synth.uniform((M, K), 87)
    Bf = synth.uniform((K, N), 88)
    assert orc.gemm_ft(Af, Bf, orc.Schedule(**DET, cadence=K // 32, level=orc.DETECT)).detected == 0
