"""Pins of the oracle's double and double-complex GEMM (Section 6 names DGEMM
and ZGEMM as the extension of the scheme) against facts the oracle cannot
produce itself: exact integer products computed with numpy int64, the real
algorithm as the special case of the complex one, the invariance of complex
norms under a rotation by i, and the unit roundoff entering the threshold."""
import numpy as np
import pytest

import oracle as orc

U64 = 2.0 ** -53


def _ints(shape, seed, lo=-8, hi=8):
    return np.random.default_rng(seed).integers(lo, hi + 1, size=shape)


def _gauss_ints(shape, seed):
    return _ints(shape, seed), _ints(shape, seed + 1000)


def _exact_complex(Ar, Ai, Br, Bi):
    """(Ar + i Ai)(Br + i Bi) in int64, real and imaginary parts apart."""
    return Ar @ Br - Ai @ Bi, Ar @ Bi + Ai @ Br


# ---- DGEMM: gemm_ft on the fp64 tiling ------------------------------------

def test_dgemm_integers_exact_and_every_target():
    M, N, K = 150, 140, 200  # ragged against the 128 x 128 tiles, 25 k-steps of 8
    A, B, Cin = _ints((M, K), 1), _ints((K, N), 2), _ints((M, N), 3)
    faults = [(0, 0, 3, 5, 7, 2.0 ** 20), (1, 1, 24, 21, 11, -3.0e5), (1, 0, 10, 4, 4, 2.0 ** 12, orc.T_ROWSUM),
              (0, 1, 12, 6, 8, -2.0 ** 14, orc.T_COLSUM)]
    res = orc.gemm_ft(A, B, orc.dgemm_schedule(cadence=4), faults=faults, alpha=2.0, beta=-1.0, Cin=Cin)
    exact = 2 * (A @ B) - Cin
    assert np.array_equal(res.C, exact.astype(np.float64))
    kinds = sorted((r.tile_m, r.tile_n, r.kind) for r in res.records)
    assert kinds == [(0, 0, 0), (0, 1, 2), (1, 0, 2), (1, 1, 0)]
    for r in res.records:
        if r.kind == 0:
            f = [f for f in faults if (f[0], f[1]) == (r.tile_m, r.tile_n)][0]
            assert r.delta == f[5] and (r.row, r.col) == (f[0] * 128 + f[3], f[1] * 128 + f[4])


def test_dgemm_period_of_detection():
    """A fault after k-step s is seen at the end of its period: the first
    multiple of the cadence at or after s + 1, or the last k-step."""
    M = N = 64
    K = 8 * 21
    A, B = _ints((M, K), 4), _ints((K, N), 5)
    for cad in (1, 4, 8):
        for s in (0, 5, 19, 20):
            res = orc.gemm_ft(A, B, orc.dgemm_schedule(cadence=cad), faults=[(0, 0, s, 3, 9, 1e6)])
            want = min(-(-(s + 1) // cad) * cad, 21) - 1
            assert [(r.kstep, r.kind) for r in res.records] == [(want, 0)]
            assert np.array_equal(res.C, (A @ B).astype(np.float64))


def test_dgemm_unit_roundoff_enters_the_threshold():
    """On N(0,1) data a relative offset of 1e-10 lies far above the
    double-precision threshold and far below a single-precision one: the fp64
    schedule detects and corrects it, one built with u = 2^-24 does not."""
    rng = np.random.default_rng(6)
    M, N, K = 96, 80, 256
    A, B = rng.standard_normal((M, K)), rng.standard_normal((K, N))
    d = 1e-10 * np.sqrt(K)
    r64 = orc.gemm_ft(A, B, orc.dgemm_schedule(cadence=8), faults=[(0, 0, 10, 7, 3, d)])
    assert [(r.row, r.col, r.kind) for r in r64.records] == [(7, 3, 0)]
    s32 = orc.dgemm_schedule(cadence=8)
    s32.u = 2.0 ** -24
    r32 = orc.gemm_ft(A, B, s32, faults=[(0, 0, 10, 7, 3, d)])
    assert r32.records == []
    exact = A @ B
    err = np.abs(r64.C - exact).max()
    assert err <= 2 * K * U64 * (np.abs(A) @ np.abs(B)).max()


def test_dgemm_no_false_alarm_on_normal_data():
    rng = np.random.default_rng(7)
    A, B = rng.standard_normal((200, 512)), rng.standard_normal((512, 180))
    res = orc.gemm_ft(A, B, orc.dgemm_schedule(cadence=1))
    assert res.detected == 0
    assert np.allclose(res.C, A @ B, rtol=0, atol=1e-11)


# ---- ZGEMM -----------------------------------------------------------------

def test_zgemm_ref_gaussian_integers_exact():
    M, N, K = 37, 29, 53
    Ar, Ai = _gauss_ints((M, K), 10)
    Br, Bi = _gauss_ints((K, N), 11)
    Cr, Ci = _gauss_ints((M, N), 12)
    alpha, beta = 2 - 1j, 1 + 3j
    got = orc.zgemm_ref(Ar + 1j * Ai, Br + 1j * Bi, alpha, beta, Cr + 1j * Ci)
    Pr, Pi = _exact_complex(Ar, Ai, Br, Bi)
    # alpha*P + beta*C, expanded by hand in integers
    wr = 2 * Pr + 1 * Pi + (1 * Cr - 3 * Ci)
    wi = 2 * Pi - 1 * Pr + (1 * Ci + 3 * Cr)
    assert np.array_equal(got.real, wr.astype(np.float64)) and np.array_equal(got.imag, wi.astype(np.float64))


def test_zgemm_ft_exact_product_and_corrections_on_both_parts():
    M, N, K = 100, 90, 120  # tiles of 64: 2 x 2, ragged; 15 k-steps of 8
    Ar, Ai = _gauss_ints((M, K), 20)
    Br, Bi = _gauss_ints((K, N), 21)
    A, B = Ar + 1j * Ai, Br + 1j * Bi
    faults = [(0, 0, 2, 3, 4, 2.0 ** 16), (0, 1, 7, 10, 20, -5000.0, orc.T_IMAG),
              (1, 0, 14, 35, 1, 777.0, orc.T_ROWSUM | orc.T_IMAG), (1, 1, 9, 2, 25, -2.0 ** 11, orc.T_COLSUM)]
    res = orc.zgemm_ft(A, B, cadence=3, faults=faults)
    Pr, Pi = _exact_complex(Ar, Ai, Br, Bi)
    assert np.array_equal(res.C.real, Pr.astype(np.float64)) and np.array_equal(res.C.imag, Pi.astype(np.float64))
    got = {(r.tile_m, r.tile_n): r for r in res.records}
    assert len(res.records) == 4
    assert got[(0, 0)].kind == 0 and got[(0, 0)].delta == 2.0 ** 16 and (got[(0, 0)].row, got[(0, 0)].col) == (3, 4)
    assert got[(0, 1)].kind == 0 and got[(0, 1)].delta == -5000j and (got[(0, 1)].row, got[(0, 1)].col) == (10, 84)
    assert got[(1, 0)].kind == 2 and got[(1, 0)].delta == 777j and got[(1, 0)].row == 99 and got[(1, 0)].col == -1
    assert got[(1, 1)].kind == 2 and got[(1, 1)].delta == -2.0 ** 11 and got[(1, 1)].col == 64 + 25
    # detection at the end of each fault's period (cadence 3, 15 k-steps)
    assert [got[k].kstep for k in ((0, 0), (0, 1), (1, 0), (1, 1))] == [2, 8, 14, 11]


def test_zgemm_two_faults_in_one_period_are_uncorrectable():
    M = N = 64
    K = 64
    Ar, Ai = _gauss_ints((M, K), 30)
    Br, Bi = _gauss_ints((K, N), 31)
    res = orc.zgemm_ft(Ar + 1j * Ai, Br + 1j * Bi, cadence=8,
                       faults=[(0, 0, 1, 3, 4, 1e5), (0, 0, 2, 9, 10, 1e5, orc.T_IMAG)])
    assert [r.kind for r in res.records] == [1]
    Pr, Pi = _exact_complex(Ar, Ai, Br, Bi)
    assert res.C[3, 4] == Pr[3, 4] + 1e5 + 1j * Pi[3, 4]
    assert res.C[9, 10] == Pr[9, 10] + 1j * (Pi[9, 10] + 1e5)


def test_zgemm_reduces_to_the_real_algorithm():
    """Imaginary parts zero: C, records and thresholds equal those of the real
    block-level algorithm on the same tiling."""
    rng = np.random.default_rng(40)
    M, N, K = 130, 70, 96
    A, B = rng.standard_normal((M, K)), rng.standard_normal((K, N))
    faults = [(0, 0, 3, 1, 2, 0.5), (2, 1, 11, 0, 5, -0.25), (1, 0, 6, 4, 4, 0.125, orc.T_COLSUM)]
    z = orc.zgemm_ft(A + 0j, B + 0j, tile=64, cadence=2, faults=faults)
    s = orc.Schedule(m_tb=64, n_tb=64, k_tb=8, m_w=64, n_w=64, m_t=8, n_t=8, cadence=2, split_k=1,
                     level=orc.BLOCK, lam=32.0, u=U64)
    r = orc.gemm_ft(A, B, s, faults=faults)
    assert np.array_equal(z.C.real, r.C) and not np.any(z.C.imag)
    assert len(z.records) == len(r.records) == 3
    for a, b in zip(z.records, r.records):
        assert (a.tile_m, a.tile_n, a.kstep, a.row, a.col, a.kind) == (b.tile_m, b.tile_n, b.kstep, b.row, b.col, b.kind)
        assert a.delta == b.delta and a.tau == b.tau


def test_zgemm_rotation_by_i():
    """A -> iA multiplies C by i and leaves every norm and threshold alone; a
    real fault rotated to an imaginary one is found at the same place with the
    same threshold.  (Norms built from a^2 instead of |a|^2 fail this.)"""
    rng = np.random.default_rng(50)
    M, N, K = 64, 64, 80
    A = rng.standard_normal((M, K)) + 1j * rng.standard_normal((M, K))
    B = rng.standard_normal((K, N)) + 1j * rng.standard_normal((K, N))
    r1 = orc.zgemm_ft(A, B, cadence=1, faults=[(0, 0, 4, 10, 20, 1e-6)])
    r2 = orc.zgemm_ft(1j * A, B, cadence=1, faults=[(0, 0, 4, 10, 20, 1e-6, orc.T_IMAG)])
    assert np.allclose(r2.C, 1j * r1.C, rtol=0, atol=1e-12)
    assert len(r1.records) == len(r2.records) == 1
    a, b = r1.records[0], r2.records[0]
    assert (a.row, a.col, a.kind) == (b.row, b.col, b.kind) == (10, 20, 0)
    assert a.tau == b.tau
    assert abs(b.delta - 1j * a.delta) <= 1e-20 + 1e-9 * abs(a.delta)


@pytest.mark.parametrize("kstep", [0, 2])
def test_zgemm_threshold_boundary_from_known_norms(kstep):
    """All entries 1 + i: |a|^2 = 2, so ||A(i,:)|| = sqrt(2K) and the block
    norms are sqrt(rows * 2K); after k = 8 (kstep + 1) elements of K a row
    checksum is k * (1 + i) * N (1 + i) = 2i k N, of modulus 2 k N.  With
    integer data the residual is exactly the offset, flagged exactly when it
    exceeds lambda * u * norms + mu * u * sqrt(k) * 2 k N."""
    M = N = 64
    K = 32
    A = np.full((M, K), 1 + 1j)
    B = np.full((K, N), 1 + 1j)
    lam, u, mu = 4.0, 2.0 ** -10, 3.0
    k = 8 * (kstep + 1)
    tau_r = lam * u * np.sqrt(2 * K) * np.sqrt(N * 2 * K) + mu * u * np.sqrt(k) * 2 * k * N
    for scale, flagged in ((0.99, False), (1.01, True)):
        res = orc.zgemm_ft(A, B, cadence=1, lam=lam, u=u, mu=mu, faults=[(0, 0, kstep, 5, 6, scale * tau_r)])
        assert (len(res.records) > 0) == flagged
        if flagged:
            assert res.records[0].kstep == kstep
            assert res.records[0].tau == pytest.approx(2 * tau_r, rel=1e-14)


@pytest.mark.parametrize("kstep,split", [(0, 1), (5, 1), (5, 2)])
def test_threshold_growth_term_from_known_checksums(kstep, split):
    """All-ones A and B (same-sign data, the case the growth term is for):
    after k elements of K in its split a tile's row checksum is k * n_tb and
    its column checksum k * m_tb, the norms are ||A(i,:)|| = sqrt(K) and
    ||B(:,J)||_F = sqrt(n_tb K).  So the row threshold is lambda * u * sqrt(K)
    * sqrt(n_tb K) + mu * u * sqrt(k) * k n_tb, and an offset on the
    accumulator is flagged exactly when it exceeds it (k-steps of 4; with two
    splits the second starts at k-step 4, so k counts from there)."""
    M = N = 16
    K = 32
    A = np.ones((M, K))
    B = np.ones((K, N))
    lam, u, mu = 2.0, 2.0 ** -12, 5.0
    s = orc.Schedule(m_tb=16, n_tb=16, k_tb=4, m_w=16, n_w=16, m_t=4, n_t=4, cadence=1, split_k=split,
                     level=orc.BLOCK, lam=lam, u=u, mu=mu)
    start = 0 if (split == 1 or kstep < 4) else 4
    k = 4 * (kstep + 1 - start)
    tau = lam * u * np.sqrt(K) * np.sqrt(16 * K) + mu * u * np.sqrt(k) * k * 16
    for scale, flagged in ((0.99, False), (1.01, True)):
        res = orc.gemm_ft(A, B, s, faults=[(0, 0, kstep, 3, 7, scale * tau)])
        assert (len(res.records) > 0) == flagged, (scale, tau)
        if flagged:
            r = res.records[0]
            assert (r.kstep, r.row, r.col, r.kind) == (kstep, 3, 7, orc.CORRECTED)
            assert r.tau == pytest.approx(2 * tau, rel=1e-12)
            assert np.max(np.abs(res.C - A @ B)) < 1e-12  # the offset came back out


def test_zgemm_no_false_alarm_and_close_to_numpy():
    rng = np.random.default_rng(60)
    A = rng.standard_normal((150, 300)) + 1j * rng.standard_normal((150, 300))
    B = rng.standard_normal((300, 110)) + 1j * rng.standard_normal((300, 110))
    res = orc.zgemm_ft(A, B, cadence=1)
    assert res.detected == 0
    assert np.abs(res.C - A @ B).max() <= 4 * 300 * U64 * (np.abs(A) @ np.abs(B)).max()
