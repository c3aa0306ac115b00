"""Python binding of libftgemm (GEMM with fused online ABFT on GB300).

Argument marshalling only: every step of the computation runs in the CUDA
kernels of ``csrc/`` behind the C ABI declared in ``include/ftgemm.h``.  The
names mirror the C entry points.  There is no CPU fallback: if the shared
library has not been built, importing the library raises.

Torch is used for device memory and streams only; matrices are passed as
device pointers taken from contiguous CUDA tensors.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass, field

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libftgemm.so")

F32, BF16, E4M3 = 0, 1, 2
FT_OFF, FT_THREAD, FT_WARP, FT_BLOCK, FT_TILE, FT_AUTO = 0, 1, 2, 3, 4, 5
LEVELS = {"off": FT_OFF, "thread": FT_THREAD, "warp": FT_WARP, "block": FT_BLOCK, "tile": FT_TILE,
          "auto": FT_AUTO}
CORRECTED, UNCORRECTABLE, CHECKSUM_ONLY = 0, 1, 2
OK, ERR_ARG, ERR_UNSUPPORTED, ERR_ALIGN, ERR_CUDA, ERR_TIMEOUT, ERR_UNRECOVERED = 0, -1, -2, -3, -4, -5, -6


class FtgemmError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"[{status}] {msg}")
        self.status = status


MLP_INPUTS = 5
MLP_PARAMS = 1281
DGEMM_TILE, ZGEMM_TILE, F64_KSTEP = 128, 64, 8
TARGET_IMAG = 4  # zgemm inject target flag: the offset is delta * i


class Schedule(C.Structure):
    """ftgemm_schedule: Table 1 tile tuple + cadence + split_k."""
    _fields_ = [("m_tb", C.c_int32), ("n_tb", C.c_int32), ("k_tb", C.c_int32),
                ("m_w", C.c_int32), ("n_w", C.c_int32), ("m_t", C.c_int32), ("n_t", C.c_int32),
                ("cadence", C.c_int32), ("split_k", C.c_int32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class InjectSpec(C.Structure):
    _fields_ = [("n", C.c_int32), ("tile_m", C.POINTER(C.c_int32)), ("tile_n", C.POINTER(C.c_int32)),
                ("kstep", C.POINTER(C.c_int32)), ("row", C.POINTER(C.c_int32)),
                ("col", C.POINTER(C.c_int32)), ("target", C.POINTER(C.c_int32)),
                ("delta", C.POINTER(C.c_float))]


class FaultRecord(C.Structure):
    _fields_ = [("tile_m", C.c_int32), ("tile_n", C.c_int32), ("kstep", C.c_int32),
                ("row", C.c_int32), ("col", C.c_int32), ("kind", C.c_int32),
                ("problem", C.c_int32), ("reserved", C.c_int32), ("delta", C.c_double), ("residual_r", C.c_double),
                ("residual_c", C.c_double), ("tau", C.c_double)]


class Problem(C.Structure):
    _fields_ = [("m", C.c_int64), ("n", C.c_int64), ("k", C.c_int64),
                ("A", C.c_void_p), ("lda", C.c_int64), ("B", C.c_void_p), ("ldb", C.c_int64),
                ("C", C.c_void_p), ("ldc", C.c_int64), ("alpha", C.c_double), ("beta", C.c_double),
                ("scale_a", C.c_float), ("scale_b", C.c_float)]


class Stats(C.Structure):
    _fields_ = [("launches", C.c_int64), ("timed_launches", C.c_int64), ("kernel_ms", C.c_double)]


class Report(C.Structure):
    _fields_ = [("detected", C.c_int64), ("corrected", C.c_int64), ("uncorrectable", C.c_int64),
                ("checksum_only", C.c_int64), ("capacity", C.c_int32), ("n_records", C.c_int32),
                ("overflow", C.c_int32), ("reserved", C.c_int32),
                ("records", C.POINTER(FaultRecord))]


@dataclass
class PyReport:
    detected: int = 0
    corrected: int = 0
    uncorrectable: int = 0
    checksum_only: int = 0
    n_records: int = 0
    overflow: bool = False
    records: list = field(default_factory=list)


_lib = None


def lib():
    """Load libftgemm.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libftgemm.so is not built ({LIB_PATH}); run "
                          "`python -c 'import __graft_entry__ as g; g.build()'`")
    L = C.CDLL(LIB_PATH)
    vp, i64, i32, dbl = C.c_void_p, C.c_int64, C.c_int32, C.c_double
    L.ftgemm_create.argtypes = [C.POINTER(vp), C.c_int, vp]
    L.ftgemm_destroy.argtypes = [vp]
    L.ftgemm_set_stream.argtypes = [vp, vp]
    L.ftgemm_set_schedule.argtypes = [vp, C.POINTER(Schedule)]
    L.ftgemm_get_schedule.argtypes = [vp, i64, i64, i64, C.c_int, C.c_int, C.POINTER(Schedule)]
    L.ftgemm_set_threshold.argtypes = [vp, C.c_int, dbl, C.POINTER(C.c_float), C.c_size_t]
    L.ftgemm_gemm.argtypes = [vp, i64, i64, i64, dbl, vp, i64, vp, i64, dbl, vp, i64, C.c_int,
                              C.c_int, C.POINTER(InjectSpec), C.POINTER(Report)]
    L.ftgemm_report_fetch.argtypes = [vp, C.POINTER(Report)]
    L.ftgemm_encode.argtypes = [vp, i64, i64, i64, vp, i64, vp, i64, i32, i32, vp, vp, vp, vp]
    L.ftgemm_set_fp8_scales.argtypes = [vp, C.c_float, C.c_float]
    L.ftgemm_quantize.argtypes = [vp, i64, vp, vp, C.c_int, C.POINTER(C.c_float)]
    L.ftgemm_enable_timing.argtypes = [vp, C.c_int]
    L.ftgemm_set_tc_pair.argtypes = [vp, C.c_int]
    L.ftgemm_autotune_tc.argtypes = [vp, i64, i64, i64, vp, i64, vp, i64, vp, i64, C.c_int, C.c_int, i32,
                                     C.POINTER(i32)]
    L.ftgemm_group_autotune.argtypes = [vp, i32, C.POINTER(Problem), C.c_int, C.c_int, i32, C.POINTER(vp),
                                        C.POINTER(i32)]
    L.ftgemm_get_stats.argtypes = [vp, C.POINTER(Stats), C.c_int]
    L.ftgemm_group_create.argtypes = [vp, i32, C.POINTER(Problem), C.c_int, C.c_int, C.POINTER(vp)]
    L.ftgemm_group_tiles.argtypes = [vp, C.POINTER(i32), C.POINTER(i32)]
    L.ftgemm_tc_tile.argtypes = [C.c_int, C.c_int, C.POINTER(i32), C.POINTER(i32)]
    L.ftgemm_group_plan.argtypes = [i32, C.POINTER(i64), C.POINTER(i64), C.POINTER(i64), C.c_int, C.c_int, i32,
                                    C.POINTER(i32), C.POINTER(i32), C.POINTER(i32)]
    L.ftgemm_group_set_faults.argtypes = [vp, C.POINTER(i32), C.POINTER(InjectSpec)]
    L.ftgemm_grouped_gemm.argtypes = [vp, vp]
    L.ftgemm_grouped_gemm_dev.argtypes = [vp, vp, i32, vp]
    L.ftgemm_group_bind_rule.argtypes = [C.POINTER(Problem), C.POINTER(Problem), C.c_int, C.c_int]
    L.ftgemm_group_destroy.argtypes = [vp]
    L.ftgemm_set_residual_sink.argtypes = [vp, vp, vp, i64]
    L.ftgemm_mlp_forward.argtypes = [vp, i64, vp, vp, vp]
    L.ftgemm_mlp_grad.argtypes = [vp, i64, vp, vp, vp, vp, C.POINTER(C.c_float)]
    L.ftgemm_mlp_train.argtypes = [vp, i64, vp, vp, i32, i32, C.c_float, vp, C.POINTER(C.c_float)]
    L.ftgemm_autotune.argtypes = [vp, i64, i64, i64, vp, i64, vp, i64, vp, i64, C.c_int, i32,
                                  C.POINTER(Schedule), C.POINTER(C.c_int)]
    L.ftgemm_selftest_wait.argtypes = [vp, i64]
    L.ftgemm_gemm_offline.argtypes = [vp, i64, i64, i64, dbl, vp, i64, vp, i64, dbl, vp, i64,
                                      C.POINTER(C.POINTER(InjectSpec)), i32, C.POINTER(i32), C.POINTER(Report)]
    L.ftgemm_gemm_nonfused.argtypes = [vp, i64, i64, i64, dbl, vp, i64, vp, i64, dbl, vp, i64, i32,
                                       C.POINTER(InjectSpec), C.POINTER(Report)]
    L.ftgemm_dgemm.argtypes = [vp, i64, i64, i64, dbl, vp, i64, vp, i64, dbl, vp, i64, C.c_int, i32,
                               C.POINTER(InjectSpec), C.POINTER(Report)]
    L.ftgemm_zgemm.argtypes = [vp, i64, i64, i64, C.POINTER(dbl), vp, i64, vp, i64, C.POINTER(dbl), vp, i64,
                               C.c_int, i32, C.POINTER(InjectSpec), C.POINTER(Report), C.POINTER(dbl)]
    L.ftgemm_status_string.argtypes = [C.c_int]
    L.ftgemm_status_string.restype = C.c_char_p
    L.ftgemm_last_error.restype = C.c_char_p
    for fn in ("ftgemm_create", "ftgemm_destroy", "ftgemm_set_stream", "ftgemm_set_schedule",
               "ftgemm_get_schedule", "ftgemm_set_threshold", "ftgemm_gemm",
               "ftgemm_report_fetch", "ftgemm_encode", "ftgemm_enable_timing", "ftgemm_set_tc_pair",
               "ftgemm_autotune_tc", "ftgemm_group_autotune",
               "ftgemm_get_stats", "ftgemm_set_fp8_scales", "ftgemm_quantize",
               "ftgemm_group_create", "ftgemm_group_plan", "ftgemm_tc_tile", "ftgemm_group_tiles", "ftgemm_group_set_faults",
               "ftgemm_grouped_gemm", "ftgemm_grouped_gemm_dev", "ftgemm_group_bind_rule",
               "ftgemm_group_destroy", "ftgemm_set_residual_sink",
               "ftgemm_mlp_forward", "ftgemm_mlp_grad", "ftgemm_mlp_train", "ftgemm_autotune",
               "ftgemm_selftest_wait", "ftgemm_gemm_offline", "ftgemm_gemm_nonfused", "ftgemm_dgemm",
               "ftgemm_zgemm"):
        getattr(L, fn).restype = C.c_int
    _lib = L
    return L


def _check(status: int):
    if status != OK:
        msg = lib().ftgemm_last_error().decode()
        raise FtgemmError(status, msg or lib().ftgemm_status_string(status).decode())


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


def _stream_ptr(stream):
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


def _records(rep: Report, cap: int) -> list:
    out = []
    for q in range(min(rep.n_records, cap)):
        r = rep.records[q]
        out.append(dict(problem=r.problem, tile_m=r.tile_m, tile_n=r.tile_n, kstep=r.kstep,
                        row=r.row, col=r.col,
                        kind=r.kind, delta=r.delta, residual_r=r.residual_r,
                        residual_c=r.residual_c, tau=r.tau))
    return out


def make_inject(faults):
    """Build an InjectSpec from tuples (tile_m, tile_n, kstep, row, col, delta[, target]).
    The returned object keeps its arrays alive."""
    n = len(faults)
    arr = {k: (C.c_int32 * max(1, n))() for k in ("tile_m", "tile_n", "kstep", "row", "col", "target")}
    dl = (C.c_float * max(1, n))()
    for q, f in enumerate(faults):
        for k, v in zip(("tile_m", "tile_n", "kstep", "row", "col"), f[:5]):
            arr[k][q] = int(v)
        dl[q] = float(f[5])
        arr["target"][q] = int(f[6]) if len(f) > 6 else 0
    spec = InjectSpec(n, arr["tile_m"], arr["tile_n"], arr["kstep"], arr["row"], arr["col"],
                      arr["target"], dl)
    spec._keep = (arr, dl)
    return spec


class Handle:
    """Owns an ftgemm handle bound to a device and a stream."""

    def __init__(self, device: int = 0, stream=None):
        import torch
        self.device = device
        with torch.cuda.device(device):
            s = _stream_ptr(stream)
        self._h = C.c_void_p()
        _check(lib().ftgemm_create(C.byref(self._h), device, s))

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib().ftgemm_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream):
        _check(lib().ftgemm_set_stream(self._h, _stream_ptr(stream)))

    def autotune_tc(self, A, B, C_out, level=FT_TILE, dtype=BF16, reps: int = 3):
        """Time single CTAs against CTA pairs for this shape (C_out is
        overwritten) and cache the faster; returns True for pairs."""
        if isinstance(level, str):
            level = LEVELS[level]
        M, K = A.shape
        N = B.shape[1]
        pick = C.c_int32(0)
        _check(lib().ftgemm_autotune_tc(self._h, M, N, K, _ptr(A), A.stride(0), _ptr(B), B.stride(0), _ptr(C_out),
                                        C_out.stride(0), dtype, level, reps, C.byref(pick)))
        return bool(pick.value)

    def set_tc_pair(self, enable):
        """Tensor-core GEMMs (and groups created later) on 2-CTA pairs (True),
        single CTAs (False), or by operand type (None, the default)."""
        _check(lib().ftgemm_set_tc_pair(self._h, -1 if enable is None else (1 if enable else 0)))

    def set_schedule(self, sched: Schedule | dict | None):
        if isinstance(sched, dict):
            sched = Schedule(**sched)
        _check(lib().ftgemm_set_schedule(self._h, C.byref(sched) if sched is not None else None))

    def get_schedule(self, m, n, k, dtype=F32, level=FT_BLOCK) -> Schedule:
        s = Schedule()
        _check(lib().ftgemm_get_schedule(self._h, m, n, k, dtype, level, C.byref(s)))
        return s

    def set_threshold(self, mode: int = 0, lam: float = 0.0, weights=None):
        w, nw = None, 0
        if weights is not None:
            import numpy as np
            wa = np.ascontiguousarray(weights, dtype=np.float32)
            w, nw = wa.ctypes.data_as(C.POINTER(C.c_float)), wa.size
        _check(lib().ftgemm_set_threshold(self._h, mode, float(lam), w, nw))

    def gemm(self, A, B, C_out, alpha=1.0, beta=0.0, level=FT_BLOCK, dtype=F32,
             inject=None, report=True, capacity: int = 4096):
        """C_out = alpha*A@B + beta*C_out through ftgemm_gemm.  A, B, C_out are
        contiguous (or row-strided) CUDA tensors; returns a PyReport if
        `report`, else None (events then accumulate in the handle)."""
        if isinstance(level, str):
            level = LEVELS[level]
        M, K = A.shape
        K2, N = B.shape
        assert K == K2 and tuple(C_out.shape) == (M, N)
        spec = make_inject(inject) if inject else None
        rep, recs = None, None
        if report:
            recs = (FaultRecord * capacity)()
            rep = Report(capacity=capacity, records=recs)
        st = lib().ftgemm_gemm(self._h, M, N, K, float(alpha), _ptr(A), A.stride(0), _ptr(B),
                               B.stride(0), float(beta), _ptr(C_out), C_out.stride(0), dtype,
                               level, C.byref(spec) if spec else None,
                               C.byref(rep) if rep else None)
        _check(st)
        if not report:
            return None
        return PyReport(rep.detected, rep.corrected, rep.uncorrectable, rep.checksum_only,
                        rep.n_records, bool(rep.overflow), _records(rep, capacity))

    def report_fetch(self, capacity: int = 4096) -> PyReport:
        recs = (FaultRecord * capacity)()
        rep = Report(capacity=capacity, records=recs)
        _check(lib().ftgemm_report_fetch(self._h, C.byref(rep)))
        return PyReport(rep.detected, rep.corrected, rep.uncorrectable, rep.checksum_only,
                        rep.n_records, bool(rep.overflow), _records(rep, capacity))

    def autotune(self, A, B, C_out, level=FT_BLOCK, reps: int = 3):
        """Time the candidate F32 schedules on these operands (C_out is
        overwritten) and cache the fastest; returns (Schedule, level)."""
        if isinstance(level, str):
            level = LEVELS[level]
        M, K = A.shape
        N = B.shape[1]
        s = Schedule()
        lv = C.c_int(0)
        _check(lib().ftgemm_autotune(self._h, M, N, K, _ptr(A), A.stride(0), _ptr(B), B.stride(0),
                                     _ptr(C_out), C_out.stride(0), level, int(reps), C.byref(s),
                                     C.byref(lv)))
        return s, lv.value

    def gemm_offline(self, A, B, C_out, alpha=1.0, beta=0.0, injects=None, max_runs: int = 8,
                     capacity: int = 4096):
        """Offline (detect-only) ABFT: attempts until one is fault-free.
        injects: one fault list per attempt (or None).  Returns (status,
        attempts, PyReport); status is OK or ERR_UNRECOVERED."""
        M, K = A.shape
        N = B.shape[1]
        specs = [make_inject(f) if f else None for f in (injects or [])]
        specs += [None] * (max_runs - len(specs))
        arr = (C.POINTER(InjectSpec) * max_runs)(*[C.pointer(sp) if sp else C.POINTER(InjectSpec)()
                                                   for sp in specs[:max_runs]])
        runs = C.c_int32(0)
        recs = (FaultRecord * capacity)()
        rep = Report(capacity=capacity, records=recs)
        st = lib().ftgemm_gemm_offline(self._h, M, N, K, float(alpha), _ptr(A), A.stride(0), _ptr(B),
                                       B.stride(0), float(beta), _ptr(C_out), C_out.stride(0), arr, max_runs,
                                       C.byref(runs), C.byref(rep))
        if st not in (OK, ERR_UNRECOVERED):
            _check(st)
        return st, runs.value, PyReport(rep.detected, rep.corrected, rep.uncorrectable, rep.checksum_only,
                                        rep.n_records, bool(rep.overflow), _records(rep, capacity))

    def dgemm(self, A, B, C_out, alpha=1.0, beta=0.0, level=FT_BLOCK, cadence: int = 16, inject=None,
              report=True, capacity: int = 4096):
        """C_out = alpha*A@B + beta*C_out in float64 through ftgemm_dgemm
        (block-level ABFT on 128 x 128 tiles, verification every `cadence`
        k-steps of 8).  Returns a PyReport if `report`, else None."""
        if isinstance(level, str):
            level = LEVELS[level]
        M, K = A.shape
        N = B.shape[1]
        assert B.shape[0] == K and tuple(C_out.shape) == (M, N)
        spec = make_inject(inject) if inject else None
        rep, recs = None, None
        if report:
            recs = (FaultRecord * capacity)()
            rep = Report(capacity=capacity, records=recs)
        _check(lib().ftgemm_dgemm(self._h, M, N, K, float(alpha), _ptr(A), A.stride(0), _ptr(B), B.stride(0),
                                  float(beta), _ptr(C_out), C_out.stride(0), level, int(cadence),
                                  C.byref(spec) if spec else None, C.byref(rep) if rep else None))
        if not report:
            return None
        return PyReport(rep.detected, rep.corrected, rep.uncorrectable, rep.checksum_only,
                        rep.n_records, bool(rep.overflow), _records(rep, capacity))

    def zgemm(self, A, B, C_out, alpha=1.0, beta=0.0, level=FT_BLOCK, cadence: int = 16, inject=None,
              report=True, capacity: int = 4096):
        """The complex128 counterpart through ftgemm_zgemm (64 x 64 tiles).
        Record fields delta / residual_r / residual_c come back as Python
        complex numbers."""
        if isinstance(level, str):
            level = LEVELS[level]
        M, K = A.shape
        N = B.shape[1]
        assert B.shape[0] == K and tuple(C_out.shape) == (M, N)
        spec = make_inject(inject) if inject else None
        al = (C.c_double * 2)(complex(alpha).real, complex(alpha).imag)
        be = (C.c_double * 2)(complex(beta).real, complex(beta).imag)
        rep, recs, im = None, None, None
        if report:
            recs = (FaultRecord * capacity)()
            rep = Report(capacity=capacity, records=recs)
            im = (C.c_double * (3 * capacity))()
        _check(lib().ftgemm_zgemm(self._h, M, N, K, al, _ptr(A), A.stride(0), _ptr(B), B.stride(0), be,
                                  _ptr(C_out), C_out.stride(0), level, int(cadence),
                                  C.byref(spec) if spec else None, C.byref(rep) if rep else None, im))
        if not report:
            return None
        rl = _records(rep, capacity)
        for q, r in enumerate(rl):
            r["delta"] = complex(r["delta"], im[3 * q])
            r["residual_r"] = complex(r["residual_r"], im[3 * q + 1])
            r["residual_c"] = complex(r["residual_c"], im[3 * q + 2])
        return PyReport(rep.detected, rep.corrected, rep.uncorrectable, rep.checksum_only,
                        rep.n_records, bool(rep.overflow), rl)

    def set_residual_sink(self, lam_needed=None, features=None):
        """Route every later TILE-level tensor-core call's and BLOCK-level
        fp32 call's per-tile residual ratios and features into the given CUDA
        tensors (None removes it)."""
        if lam_needed is None:
            _check(lib().ftgemm_set_residual_sink(self._h, None, None, 0))
            return
        assert features.numel() == MLP_INPUTS * lam_needed.numel()
        _check(lib().ftgemm_set_residual_sink(self._h, _ptr(lam_needed), _ptr(features),
                                              lam_needed.numel()))

    def mlp_forward(self, X, theta):
        import torch
        y = torch.empty(X.shape[0], dtype=torch.float32, device=X.device)
        _check(lib().ftgemm_mlp_forward(self._h, X.shape[0], _ptr(X), _ptr(theta), _ptr(y)))
        return y

    def mlp_grad(self, X, t, theta):
        """(loss, gradient tensor) of the mean squared error."""
        import torch
        g = torch.empty(MLP_PARAMS, dtype=torch.float32, device=X.device)
        L = C.c_float(0.0)
        _check(lib().ftgemm_mlp_grad(self._h, X.shape[0], _ptr(X), _ptr(t), _ptr(theta), _ptr(g),
                                     C.byref(L)))
        return L.value, g

    def mlp_train(self, X, t, theta, epochs: int, batch: int, lr: float):
        """Minibatch Adam on the GPU, in place on theta; returns the mean
        loss of each epoch."""
        out = (C.c_float * epochs)()
        _check(lib().ftgemm_mlp_train(self._h, X.shape[0], _ptr(X), _ptr(t), int(epochs), int(batch),
                                      float(lr), _ptr(theta), out))
        return list(out)

    def set_fp8_scales(self, scale_a: float, scale_b: float):
        _check(lib().ftgemm_set_fp8_scales(self._h, float(scale_a), float(scale_b)))

    def quantize(self, x, dtype=BF16):
        """Quantize a contiguous fp32 CUDA tensor to bf16 (torch.bfloat16) or
        E4M3 codes (torch.uint8).  Returns (y, scale)."""
        import torch
        if dtype == BF16:
            y = torch.empty(x.shape, dtype=torch.bfloat16, device=x.device)
        else:
            y = torch.empty(x.shape, dtype=torch.uint8, device=x.device)
        sc = C.c_float(0.0)
        _check(lib().ftgemm_quantize(self._h, x.numel(), _ptr(x), _ptr(y), dtype, C.byref(sc)))
        return y, sc.value

    def enable_timing(self, enable: bool = True):
        _check(lib().ftgemm_enable_timing(self._h, 1 if enable else 0))

    def stats(self, reset: bool = False) -> dict:
        st = Stats()
        _check(lib().ftgemm_get_stats(self._h, C.byref(st), 1 if reset else 0))
        return dict(launches=st.launches, timed_launches=st.timed_launches, kernel_ms=st.kernel_ms)

    def encode(self, A, B, m_u, n_u, V=None, W=None, nA=None, nB=None):
        M, K = A.shape
        _, N = B.shape
        _check(lib().ftgemm_encode(self._h, M, N, K, _ptr(A), A.stride(0), _ptr(B), B.stride(0),
                                   m_u, n_u, _ptr(V), _ptr(W), _ptr(nA), _ptr(nB)))


def tc_tile(dtype=BF16, level=FT_TILE):
    """(rows, cols) of the data tile of C one tensor-core CTA computes and
    verifies (ftgemm_tc_tile): 128 x 256 at level OFF; at TILE 125 x 248 for
    bf16 and 123 x 248 for e4m3.  Fault tile indices and in-tile offsets
    refer to this grid."""
    r, c = C.c_int32(0), C.c_int32(0)
    _check(lib().ftgemm_tc_tile(dtype, level, C.byref(r), C.byref(c)))
    return r.value, c.value


def group_plan(shapes, dtype=BF16, level=FT_TILE, ncta: int = 152):
    """The static tile schedule ftgemm_group_create would build for problems
    of sizes shapes = [(m, n, k), ...] over `ncta` persistent CTAs, computed
    on the host (ftgemm_group_plan).  Returns (tiles, cta_start): tiles is a
    list of (problem, tile_m, tile_n, k_blocks) listed CTA by CTA, and CTA c
    runs tiles[cta_start[c]:cta_start[c + 1]]."""
    count = len(shapes)
    m = (C.c_int64 * max(1, count))(*[s[0] for s in shapes])
    n = (C.c_int64 * max(1, count))(*[s[1] for s in shapes])
    k = (C.c_int64 * max(1, count))(*[s[2] for s in shapes])
    total = C.c_int32(0)
    _check(lib().ftgemm_group_plan(count, m, n, k, dtype, level, ncta, None, None, C.byref(total)))
    tiles = (C.c_int32 * (4 * max(1, total.value)))()
    start = (C.c_int32 * (ncta + 1))()
    _check(lib().ftgemm_group_plan(count, m, n, k, dtype, level, ncta, tiles, start, C.byref(total)))
    flat = list(tiles)[:4 * total.value]
    return [tuple(flat[i:i + 4]) for i in range(0, len(flat), 4)], list(start)


def problem_structs(problems):
    """ftgemm_problem structs (host) of (A, B, C[, alpha, beta[, scale_a,
    scale_b]]) tuples of CUDA tensors."""
    arr = (Problem * len(problems))()
    for q, pr in enumerate(problems):
        A, B, Cm = pr[:3]
        alpha = float(pr[3]) if len(pr) > 3 else 1.0
        beta = float(pr[4]) if len(pr) > 4 else 0.0
        sa = float(pr[5]) if len(pr) > 5 else 1.0
        sb = float(pr[6]) if len(pr) > 6 else 1.0
        m, k = A.shape
        n = B.shape[1]
        arr[q] = Problem(m, n, k, A.data_ptr(), A.stride(0), B.data_ptr(), B.stride(0),
                         Cm.data_ptr(), Cm.stride(0), alpha, beta, sa, sb)
    return arr


def problem_table(problems, device="cuda"):
    """The ftgemm_problem array of `problems` (as for Group) copied into a
    device tensor (int64 words), for Group.run_device."""
    import torch
    arr = problem_structs(problems)
    host = torch.frombuffer(bytearray(bytes(arr)), dtype=torch.int64)
    return host.to(device)


def bind_rule(created, bound, dtype=BF16, level=FT_TILE):
    """ftgemm_group_bind_rule on two Problem structs (host only)."""
    return lib().ftgemm_group_bind_rule(C.byref(created), C.byref(bound), dtype, level)


class Group:
    """A prepared group of tensor-core GEMMs (ftgemm_group_create).

    problems: list of (A, B, C) CUDA tensors, or (A, B, C, alpha, beta[,
    scale_a, scale_b]); A m x k and B k x n of `dtype` (bf16 tensors, or
    uint8 E4M3 codes), C fp32 m x n.  The tensors must outlive the group."""

    def __init__(self, handle: "Handle", problems, dtype=BF16, level=FT_TILE, tune: int = 0):
        """tune > 0: the schedule (single CTAs or CTA pairs) is chosen by
        running the group both ways in `tune` interleaved rounds (every C is
        overwritten); self.pair tells which."""
        self.handle = handle
        self.count = len(problems)
        arr = problem_structs(problems)
        self._keep = list(problems)
        self._g = C.c_void_p()
        self.pair = None
        if tune > 0:
            pick = C.c_int32(0)
            _check(lib().ftgemm_group_autotune(handle._h, self.count, arr, dtype, level, tune, C.byref(self._g),
                                               C.byref(pick)))
            self.pair = bool(pick.value)
        else:
            _check(lib().ftgemm_group_create(handle._h, self.count, arr, dtype, level, C.byref(self._g)))

    def tiles(self):
        tm = (C.c_int32 * self.count)()
        tn = (C.c_int32 * self.count)()
        _check(lib().ftgemm_group_tiles(self._g, tm, tn))
        return list(tm), list(tn)

    def set_faults(self, faults):
        """faults: tuples (problem, tile_m, tile_n, kstep, row, col, delta[, target])."""
        if not faults:
            _check(lib().ftgemm_group_set_faults(self._g, None, None))
            return
        prob = (C.c_int32 * len(faults))(*[int(f[0]) for f in faults])
        spec = make_inject([tuple(f[1:]) for f in faults])
        _check(lib().ftgemm_group_set_faults(self._g, prob, C.byref(spec)))

    def run(self):
        """Enqueue the whole group on the handle's stream (no host sync)."""
        _check(lib().ftgemm_grouped_gemm(self.handle._h, self._g))

    def run_device(self, table):
        """Enqueue the group with its operands read from `table`, a CUDA
        tensor holding `count` ftgemm_problem structs (problem_table), when
        the call runs on the stream (ftgemm_grouped_gemm_dev).  The tensors it
        points at must outlive every launch that reads them."""
        assert table.is_cuda and table.numel() * table.element_size() >= self.count * C.sizeof(Problem)
        _check(lib().ftgemm_grouped_gemm_dev(self.handle._h, self._g, self.count, C.c_void_p(table.data_ptr())))

    def close(self):
        if getattr(self, "_g", None) and self._g.value:
            lib().ftgemm_group_destroy(self._g)
            self._g = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
