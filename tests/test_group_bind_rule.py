"""The rebinding rule of ftgemm_grouped_gemm_dev, on the host: the same
function the rebinding kernel runs on each entry of the device array, called
through ftgemm_group_bind_rule with made-up addresses (nothing is read at
them; no GPU needed).  Every rule, each broken alone, and the order in which
they are checked."""
import pytest

BASE = dict(m=300, n=500, k=256, A=0x7F0000100000, lda=256, B=0x7F0000200000, ldb=512,
            C=0x7F0000300000, ldc=500, alpha=1.0, beta=0.0, scale_a=1.0, scale_b=1.0)


@pytest.fixture(scope="module")
def ft():
    import paper_2305_01024_gb300 as ft
    ft.lib()
    return ft


def _p(ft, **kw):
    d = dict(BASE)
    d.update(kw)
    return ft.Problem(**d)


def test_the_creation_entry_itself_passes(ft):
    for dt in (ft.BF16, ft.E4M3):
        for lv in (ft.FT_OFF, ft.FT_TILE):
            assert ft.bind_rule(_p(ft), _p(ft), dt, lv) == 0
    # new operands, C, ldc, alpha, beta are free
    moved = _p(ft, A=0x7F0000500010, B=0x7F0000600002, C=0x7F0000700004, ldc=640, alpha=-2.0, beta=0.5)
    assert ft.bind_rule(_p(ft), moved, ft.BF16, ft.FT_TILE) == 0


@pytest.mark.parametrize("field,value,code", [
    ("m", 301, 1), ("n", 499, 1), ("k", 264, 1),
    ("lda", 264, 2), ("ldb", 520, 2),
    ("A", 0, 3), ("B", 0, 3), ("C", 0, 3),
    ("A", 0x7F0000100008, 4),
    ("B", 0x7F0000200001, 5),
    ("ldc", 499, 6), ("C", 0x7F0000300002, 6),
])
def test_each_rule_broken_alone(ft, field, value, code):
    assert ft.bind_rule(_p(ft), _p(ft, **{field: value}), ft.BF16, ft.FT_TILE) == code


def test_b_read_in_place_needs_16_bytes(ft):
    # bf16 at level OFF with a 16-byte aligned B and row stride: the MMA reads
    # B in place, so a rebound B must be 16-byte aligned too
    created = _p(ft)  # ldb 512 elements = 1024 bytes
    assert ft.bind_rule(created, _p(ft, B=0x7F0000200008), ft.BF16, ft.FT_OFF) == 5
    # with checksums B goes through B^T: element alignment is enough
    assert ft.bind_rule(created, _p(ft, B=0x7F0000200008), ft.BF16, ft.FT_TILE) == 0
    # a created B that was not 16-byte aligned was never read in place
    created_odd = _p(ft, B=0x7F0000200002)
    assert ft.bind_rule(created_odd, _p(ft, B=0x7F0000200008), ft.BF16, ft.FT_OFF) == 0
    # e4m3 elements are bytes: any address
    assert ft.bind_rule(created, _p(ft, B=0x7F0000200001), ft.E4M3, ft.FT_TILE) == 0


@pytest.mark.parametrize("sa,sb", [(0.0, 1.0), (1.0, -1.0), (float("nan"), 1.0), (1e30, 1e30), (float("inf"), 1.0)])
def test_e4m3_scales(ft, sa, sb):
    assert ft.bind_rule(_p(ft), _p(ft, scale_a=sa, scale_b=sb), ft.E4M3, ft.FT_TILE) == 7
    # bf16 ignores the scales
    assert ft.bind_rule(_p(ft), _p(ft, scale_a=sa, scale_b=sb), ft.BF16, ft.FT_TILE) == 0


def test_rules_are_checked_in_order(ft):
    # sizes before leading dimensions before NULL before alignment
    assert ft.bind_rule(_p(ft), _p(ft, m=1, lda=1, A=0), ft.BF16, ft.FT_TILE) == 1
    assert ft.bind_rule(_p(ft), _p(ft, lda=1, A=0), ft.BF16, ft.FT_TILE) == 2
    assert ft.bind_rule(_p(ft), _p(ft, A=0, C=0x7F0000300002), ft.BF16, ft.FT_TILE) == 3


def test_unsupported_combinations_are_errors(ft):
    assert ft.bind_rule(_p(ft), _p(ft), ft.F32, ft.FT_TILE) == ft.ERR_UNSUPPORTED
    assert ft.bind_rule(_p(ft), _p(ft), ft.BF16, ft.FT_BLOCK) == ft.ERR_UNSUPPORTED
