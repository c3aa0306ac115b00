"""CPU FP64 oracle for fused online-ABFT GEMM (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA library
``paper_2305_01024_gb300``; the two meet only through the seeded inputs of
``synth``.  The arithmetic lives in ``ftgemm_oracle.c`` (plain C, double
precision, OpenMP over output tiles); this module only marshals numpy arrays.

Functions (each cites the paper passage it follows):
  gemm_ref      plain definition C = alpha*A*B + beta*C_in (Section 3.1)
  encode        e^T A per row block, B e per column block (Eq. 1-2) and norms
  gemm_ft       the online ABFT algorithm: Eq. 4 checksums, periodic
                verification, location and correction (Sections 2.2, 4.2)
  dgemm_schedule  the fp64 (DGEMM) tiling: gemm_ft with u = 2^-53 (Section 6)
  zgemm_ref / zgemm_ft  the same on complex values (Section 6: ZGEMM)
  round_bf16    RNE rounding to bfloat16
  quant_e4m3    per-tensor amax scaling + RNE/saturating E4M3 (OCP FP8)
  offline_expected_runs  online vs offline ABFT cost model (Section 5.5)
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ftgemm_oracle.c")
_OUT = os.path.join(_HERE, "_build", "libftgemm_oracle.so")

OFF, THREAD, WARP, BLOCK, TILE, DETECT = 0, 1, 2, 3, 4, 5
# threshold scales: lambda for the norm term, mu for the checksum-growth term
LAM = 32.0
MU = 8.0
CORRECTED, UNCORRECTABLE, CHECKSUM_ONLY = 0, 1, 2
T_ACC, T_ROWSUM, T_COLSUM = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, OpenMP) into oracle/_build/."""
    if not force and os.path.exists(_OUT) and os.path.getmtime(_OUT) >= os.path.getmtime(_SRC):
        return _OUT
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    tmp = _OUT + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", "-o", tmp, _SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _OUT)
    return _OUT


class _Sched(C.Structure):
    _fields_ = [("m_tb", C.c_int32), ("n_tb", C.c_int32), ("k_tb", C.c_int32),
                ("m_w", C.c_int32), ("n_w", C.c_int32), ("m_t", C.c_int32), ("n_t", C.c_int32),
                ("cadence", C.c_int32), ("split_k", C.c_int32), ("level", C.c_int32),
                ("lam", C.c_double), ("u", C.c_double), ("mu", C.c_double)]


class _Fault(C.Structure):
    _fields_ = [("tile_m", C.c_int32), ("tile_n", C.c_int32), ("kstep", C.c_int32),
                ("row", C.c_int32), ("col", C.c_int32), ("target", C.c_int32),
                ("delta", C.c_double)]


class _ZRec(C.Structure):
    _fields_ = [("tile_m", C.c_int32), ("tile_n", C.c_int32), ("kstep", C.c_int32),
                ("row", C.c_int32), ("col", C.c_int32), ("kind", C.c_int32),
                ("delta_re", C.c_double), ("delta_im", C.c_double),
                ("res_r_re", C.c_double), ("res_r_im", C.c_double),
                ("res_c_re", C.c_double), ("res_c_im", C.c_double), ("tau", C.c_double)]


class _Rec(C.Structure):
    _fields_ = [("tile_m", C.c_int32), ("tile_n", C.c_int32), ("kstep", C.c_int32),
                ("row", C.c_int32), ("col", C.c_int32), ("kind", C.c_int32),
                ("delta", C.c_double), ("residual_r", C.c_double),
                ("residual_c", C.c_double), ("tau", C.c_double)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        d, i64, i32 = C.POINTER(C.c_double), C.c_int64, C.c_int32
        _lib.orc_gemm_ref.argtypes = [i64, i64, i64, C.c_double, d, i64, d, i64,
                                      C.c_double, d, i64, d, i64]
        _lib.orc_encode.argtypes = [i64, i64, i64, d, i64, d, i64, i32, i32, d, d, d, d]
        _lib.orc_gemm_ft.argtypes = [i64, i64, i64, C.c_double, d, i64, d, i64, C.c_double,
                                     d, i64, d, i64, C.POINTER(_Sched), C.POINTER(_Fault),
                                     i32, C.POINTER(_Rec), i32, C.POINTER(C.c_int64),
                                     C.POINTER(C.c_int32)]
        _lib.orc_gemm_ft.restype = C.c_int
        _lib.orc_zgemm_ref.argtypes = [i64, i64, i64, d, d, i64, d, i64, d, d, i64, d, i64]
        _lib.orc_zgemm_ft.argtypes = [i64, i64, i64, d, d, i64, d, i64, d, d, i64, d, i64,
                                      i32, i32, i32, i32, i32, C.c_double, C.c_double, C.c_double,
                                      C.POINTER(_Fault), i32, C.POINTER(_ZRec), i32,
                                      C.POINTER(C.c_int64), C.POINTER(C.c_int32)]
        _lib.orc_zgemm_ft.restype = C.c_int
        _lib.orc_round_bf16.argtypes = [C.POINTER(C.c_float), i64, d]
        _lib.orc_quant_e4m3.argtypes = [C.POINTER(C.c_float), i64, d, d]
        _lib.orc_quant_e4m3.restype = C.c_double
        _lib.orc_offline_expected_runs.argtypes = [C.c_double, C.c_double]
        _lib.orc_offline_expected_runs.restype = C.c_double
        _lib.orc_num_threads.restype = C.c_int
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def num_threads() -> int:
    return int(lib().orc_num_threads())


@dataclass
class Schedule:
    """Tiling and checksum schedule (Table 1 tuple + verification cadence)."""
    m_tb: int = 128
    n_tb: int = 128
    k_tb: int = 8
    m_w: int = 32
    n_w: int = 64
    m_t: int = 8
    n_t: int = 8
    cadence: int = 32
    split_k: int = 1
    level: int = BLOCK
    lam: float = LAM
    u: float = 2.0 ** -24
    mu: float = MU


@dataclass
class Record:
    tile_m: int
    tile_n: int
    kstep: int
    row: int
    col: int
    kind: int
    delta: float
    residual_r: float
    residual_c: float
    tau: float


@dataclass
class Result:
    C: np.ndarray
    detected: int
    corrected: int
    uncorrectable: int
    checksum_only: int
    records: list


def gemm_ref(A, B, alpha=1.0, beta=0.0, Cin=None) -> np.ndarray:
    """C = alpha*A*B + beta*C_in, every product and sum in double precision
    (the problem of Section 3.1)."""
    A, B = _f64(A), _f64(B)
    M, K = A.shape
    K2, N = B.shape
    assert K == K2
    Ci = _f64(Cin) if (Cin is not None and beta != 0.0) else np.zeros((1, 1))
    out = np.empty((M, N), dtype=np.float64)
    lib().orc_gemm_ref(M, N, K, alpha, _dp(A), K, _dp(B), N, beta, _dp(Ci),
                       Ci.shape[1] if Ci.ndim == 2 else 1, _dp(out), N)
    return out


def encode(A, B, m_u: int, n_u: int):
    """Eq. 1-2 per block: return V (row-block sums of A, [blocks][K]), W (column-block sums of B,
    [blocks][K]), nA (row 2-norms of A), nB (column 2-norms of B)."""
    A, B = _f64(A), _f64(B)
    M, K = A.shape
    _, N = B.shape
    mb, nb = -(-M // m_u), -(-N // n_u)
    V = np.empty((mb, K)); W = np.empty((nb, K)); nA = np.empty(M); nB = np.empty(N)
    lib().orc_encode(M, N, K, _dp(A), K, _dp(B), N, m_u, n_u, _dp(V), _dp(W), _dp(nA), _dp(nB))
    return V, W, nA, nB


def gemm_ft(A, B, sched: Schedule, faults=(), alpha=1.0, beta=0.0, Cin=None,
            cap: int = 1 << 16) -> Result:
    """Run the online ABFT GEMM of the paper on the CPU.

    ``faults`` is a sequence of (tile_m, tile_n, kstep, row, col, delta[, target])
    with tile-local row/col; kstep -1 means the last k-step.
    """
    A, B = _f64(A), _f64(B)
    M, K = A.shape
    K2, N = B.shape
    assert K == K2
    Ci = _f64(Cin) if (Cin is not None and beta != 0.0) else np.zeros((1, 1))
    out = np.empty((M, N), dtype=np.float64)
    s = _Sched(sched.m_tb, sched.n_tb, sched.k_tb, sched.m_w, sched.n_w, sched.m_t,
               sched.n_t, sched.cadence, sched.split_k, sched.level, sched.lam, sched.u, sched.mu)
    nf = len(faults)
    fa = (_Fault * max(1, nf))()
    for q, f in enumerate(faults):
        tgt = f[6] if len(f) > 6 else T_ACC
        fa[q] = _Fault(int(f[0]), int(f[1]), int(f[2]), int(f[3]), int(f[4]), int(tgt), float(f[5]))
    recs = (_Rec * cap)()
    cnt = (C.c_int64 * 4)()
    nrec = C.c_int32(0)
    rc = lib().orc_gemm_ft(M, N, K, alpha, _dp(A), K, _dp(B), N, beta, _dp(Ci),
                           Ci.shape[1], _dp(out), N, C.byref(s), fa, nf, recs, cap,
                           cnt, C.byref(nrec))
    if rc != 0:
        raise ValueError(f"orc_gemm_ft rejected its arguments (rc={rc})")
    rl = [Record(r.tile_m, r.tile_n, r.kstep, r.row, r.col, r.kind, r.delta,
                 r.residual_r, r.residual_c, r.tau) for r in recs[: min(nrec.value, cap)]]
    return Result(out, cnt[0], cnt[1], cnt[2], cnt[3], rl)


U64 = 2.0 ** -53
T_IMAG = 4  # fault target flag of the complex GEMM: the offset is delta * i


def dgemm_schedule(cadence: int, lam: float = LAM, level: int = BLOCK, mu: float = MU) -> Schedule:
    """The double-precision GEMM's tiling for gemm_ft (DGEMM, the extension
    Section 6 names): 128 x 128 output tiles, k-steps of 8, one verification
    unit per tile, u = 2^-53."""
    return Schedule(m_tb=128, n_tb=128, k_tb=8, m_w=128, n_w=128, m_t=8, n_t=8, cadence=cadence,
                    split_k=1, level=level, lam=lam, u=U64, mu=mu)


def _c128(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.complex128))


def zgemm_ref(A, B, alpha=1.0, beta=0.0, Cin=None) -> np.ndarray:
    """C = alpha*A*B + beta*C_in in complex double precision (the plain
    definition behind Section 6's ZGEMM)."""
    A, B = _c128(A), _c128(B)
    M, K = A.shape
    K2, N = B.shape
    assert K == K2
    Ci = _c128(Cin) if (Cin is not None and beta != 0) else np.zeros((1, 1), np.complex128)
    out = np.empty((M, N), dtype=np.complex128)
    al = np.array([complex(alpha).real, complex(alpha).imag])
    be = np.array([complex(beta).real, complex(beta).imag])
    lib().orc_zgemm_ref(M, N, K, _dp(al), _dp(A), K, _dp(B), N, _dp(be), _dp(Ci), Ci.shape[1], _dp(out), N)
    return out


@dataclass
class ZRecord:
    tile_m: int
    tile_n: int
    kstep: int
    row: int
    col: int
    kind: int
    delta: complex
    residual_r: complex
    residual_c: complex
    tau: float


def zgemm_ft(A, B, tile: int = 64, k_tb: int = 8, cadence: int = 1, faults=(), alpha=1.0, beta=0.0,
             Cin=None, lam: float = LAM, u: float = U64, verify: bool = True, mu: float = MU,
             cap: int = 1 << 16) -> Result:
    """The online ABFT GEMM on complex operands at block level (ZGEMM, the
    extension Section 6 names; the steps of gemm_ft on complex values): tile x tile
    output tiles, k-steps of k_tb, verification every `cadence` k-steps.
    ``faults``: (tile_m, tile_n, kstep, row, col, delta[, target]) with a real
    delta; target | T_IMAG puts the offset on the imaginary part."""
    A, B = _c128(A), _c128(B)
    M, K = A.shape
    K2, N = B.shape
    assert K == K2
    Ci = _c128(Cin) if (Cin is not None and beta != 0) else np.zeros((1, 1), np.complex128)
    out = np.empty((M, N), dtype=np.complex128)
    al = np.array([complex(alpha).real, complex(alpha).imag])
    be = np.array([complex(beta).real, complex(beta).imag])
    nf = len(faults)
    fa = (_Fault * max(1, nf))()
    for q, f in enumerate(faults):
        tgt = f[6] if len(f) > 6 else T_ACC
        fa[q] = _Fault(int(f[0]), int(f[1]), int(f[2]), int(f[3]), int(f[4]), int(tgt), float(f[5]))
    recs = (_ZRec * cap)()
    cnt = (C.c_int64 * 4)()
    nrec = C.c_int32(0)
    rc = lib().orc_zgemm_ft(M, N, K, _dp(al), _dp(A), K, _dp(B), N, _dp(be), _dp(Ci), Ci.shape[1],
                            _dp(out), N, tile, tile, k_tb, cadence, 1 if verify else 0, lam, u, mu,
                            fa, nf, recs, cap, cnt, C.byref(nrec))
    if rc != 0:
        raise ValueError(f"orc_zgemm_ft rejected its arguments (rc={rc})")
    rl = [ZRecord(r.tile_m, r.tile_n, r.kstep, r.row, r.col, r.kind, complex(r.delta_re, r.delta_im),
                  complex(r.res_r_re, r.res_r_im), complex(r.res_c_re, r.res_c_im), r.tau)
          for r in recs[: min(nrec.value, cap)]]
    return Result(out, cnt[0], cnt[1], cnt[2], cnt[3], rl)


def round_bf16(x) -> np.ndarray:
    """Round fp32 values to bfloat16, nearest with ties to even (the bf16
    format; no counterpart in the paper, whose kernels are fp32)."""
    x = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    out = np.empty(x.shape, dtype=np.float64)
    lib().orc_round_bf16(x.ctypes.data_as(C.POINTER(C.c_float)), x.size, _dp(out))
    return out


def quant_e4m3(x):
    """Per-tensor amax scaling and saturating round-to-nearest-even to OCP FP8
    E4M3 (no counterpart in the paper, whose kernels are fp32).  Return
    (dequantized values, raw E4M3 values, scale)."""
    x = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    out = np.empty(x.shape, dtype=np.float64)
    q = np.empty(x.shape, dtype=np.float64)
    s = lib().orc_quant_e4m3(x.ctypes.data_as(C.POINTER(C.c_float)), x.size, _dp(out), _dp(q))
    return out, q, s


def offline_expected_runs(gamma0: float, tiles: float) -> float:
    """Expected runs of offline (detect-and-restart) ABFT, Section 5.5:
    (1 - gamma) / (1 - 2 gamma) with gamma = 1 - (1 - gamma0)^tiles; infinite
    for gamma >= 1/2."""
    return float(lib().orc_offline_expected_runs(gamma0, tiles))
