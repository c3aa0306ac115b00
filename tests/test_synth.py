"""The seeded input generators that the oracle, the GPU tests and bench.py
share: the splitmix64 stream against the reference outputs of its published
definition, the device-side torch twin bit for bit against numpy, sub-blocks
against the full matrix, each family's value set and moments, and the
invariants of the fault draws.  CPU only."""
import numpy as np
import pytest

import synth


def test_splitmix64_reference_outputs():
    # splitmix64 (Steele, Lea and Flood, OOPSLA 2014) started from state 0
    # yields e220a8397b1dcdaf, 6e789e6aa1b965f4, 06c45d188009454f; element 0
    # of stream s is the generator's output number s
    want = [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    assert [int(synth.raw_u64(s, 1)[0]) for s in range(3)] == want


def test_counter_based_offsets():
    a = synth.raw_u64(77, 1000)
    b = synth.raw_u64(77, 300, offset=700)
    assert np.array_equal(a[700:], b)
    assert not np.array_equal(synth.raw_u64(78, 300, offset=700), b)


def test_unit_range_and_resolution():
    u = synth.unit(5, 1 << 16)
    assert u.min() >= 0.0 and u.max() < 1.0
    assert np.all(u * 2.0 ** 53 == np.floor(u * 2.0 ** 53))  # 53 random bits, exact


@pytest.mark.parametrize("kind", ["int", "uniform", "normal"])
def test_torch_twin_matches_numpy(kind):
    pytest.importorskip("torch")
    shape = (37, 129)
    a = synth.make(kind, shape, 4242)
    b = synth.torch_make(kind, shape, 4242, "cpu").numpy()
    assert b.dtype == np.float32 and b.shape == shape
    if kind == "normal":  # the two libraries' log1p and cos may differ in the last bit
        np.testing.assert_allclose(b, a, rtol=1e-6, atol=1e-6)
    else:
        assert np.array_equal(a, b)


def test_block_is_a_slice_of_the_full_matrix():
    for kind in ("int", "uniform", "normal"):
        full = synth.make(kind, (50, 70), 99)
        sub = synth.block(kind, 99, (50, 70), (7, 31), (13, 70))
        assert np.array_equal(sub, full[7:31, 13:70])


def test_integer_family_values_and_frequencies():
    v = synth.integers((90000,), 1)
    vals, counts = np.unique(v, return_counts=True)
    assert list(vals) == list(range(-4, 5))
    n, p = v.size, 1.0 / 9.0
    assert np.all(np.abs(counts - n * p) < 5 * np.sqrt(n * p * (1 - p)))


def test_uniform_and_normal_moments():
    u = synth.uniform((200000,), 2).astype(np.float64)
    assert u.min() >= -1.0 and u.max() < 1.0
    assert abs(u.mean()) < 5 * np.sqrt(1.0 / 3.0 / u.size)
    assert abs(u.var() - 1.0 / 3.0) < 0.01
    z = synth.normal((200000,), 3).astype(np.float64)
    assert abs(z.mean()) < 5 / np.sqrt(z.size)
    assert abs(z.std() - 1.0) < 0.01
    assert abs(np.mean(np.abs(z) > 3.0) - 0.0027) < 0.001  # two-sided 3-sigma tail


def test_fault_positions_in_bounds_distinct_and_reproducible():
    M, N, m_tb, n_tb, ksteps, cadence = 1000, 777, 128, 128, 64, 8
    tiles_m, tiles_n = -(-M // m_tb), -(-N // n_tb)
    args = (11, 200, tiles_m, tiles_n, ksteps, m_tb, n_tb, M, N, cadence)
    pos = synth.fault_positions(*args)
    assert len(pos) == 200
    units = set()
    for tm, tn, ks, r, c in pos:
        assert 0 <= tm < tiles_m and 0 <= tn < tiles_n and 0 <= ks < ksteps
        assert 0 <= r < m_tb and 0 <= c < n_tb
        assert tm * m_tb + r < M and tn * n_tb + c < N  # inside the ragged edge tiles too
        units.add((tm, tn, ks // cadence))
    assert len(units) == len(pos)  # at most one fault per tile and period
    assert synth.fault_positions(*args) == pos


def test_fault_positions_with_thread_units():
    # with a finer verification unit two faults may share a tile and period,
    # but never a unit
    unit_of = lambda r, c: (r // 16, c // 8)
    pos = synth.fault_positions(12, 300, 2, 2, 4, 128, 128, 256, 256, 4, unit_of=unit_of)
    keys = {(tm, tn, ks // 4, unit_of(r, c)) for tm, tn, ks, r, c in pos}
    assert len(keys) == len(pos)
    assert len({(tm, tn, ks // 4) for tm, tn, ks, _, _ in pos}) < len(pos)


def test_poisson_and_log_uniform_draws():
    lam = 3.5
    ks = np.array([synth.poisson(5, lam, i) for i in range(20000)], dtype=np.float64)
    assert abs(ks.mean() - lam) < 5 * np.sqrt(lam / ks.size)
    assert abs(ks.var() - lam) < 0.15
    assert synth.poisson(5, 0.0) == 0
    g = synth.log_uniform(6, 100000, 1e-2, 1e3)
    assert g.min() >= 1e-2 and g.max() <= 1e3
    assert abs(np.log10(g).mean() - 0.5) < 0.02  # log10 uniform on [-2, 3]
