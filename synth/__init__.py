"""Seeded synthetic inputs shared by the oracle harness, the GPU tests and bench.py.

This module holds no ABFT arithmetic: it only turns (seed, index) into numbers.
The generator is counter based: element ``i`` of stream ``seed`` is the
splitmix64 output function (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014) applied to the state
``seed*phi + i + phi`` (mod 2^64, phi = 0x9E3779B97F4A7C15), so any
element can be produced independently, in numpy on the host or in torch on a
device, with identical bits for the uniform and integer families.

Distributions (the shapes the paper's experiments use, Section 5):
  * ``integers``  floor(9u) - 4, i.e. uniform on {-4..4}; exact in fp32 GEMMs
  * ``uniform``   2u - 1 on [-1, 1)
  * ``normal``    Box-Muller from two independent streams (host libm)

Random choices of the method's test harness (fault positions and magnitudes)
are also drawn here and then passed to both the oracle and the CUDA path.
"""
from __future__ import annotations

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
BASE_SEED = 2305_01024


# Each workload draws its inputs from its own block of 100 streams.
WORKLOADS = {
    "int256": 1,          # 256^3 integer-valued fp32, block level, 4 faults of 2^10
    "sweep_fp32": 2,      # square fp32 sweep 1024..16384, U(-1,1), beta = 0.5
    "irregular_fp32": 3,  # five irregular fp32 shapes, N(0,1)
    "tc_square": 4,       # bf16 / e4m3 squares 4096..16384, N(0,1)
    "group512": 5,        # 512 bf16 problems, M, N on 64..4096, K on 64..2048
    "dgemm": 6,           # fp64 DGEMM, N(0,1)
    "zgemm": 7,           # complex fp64 ZGEMM, N(0,1)
}


def workload_seed(workload: str, index: int) -> int:
    """Seed of input ``index`` of a named workload (seed = 230501024 + 100*block + index)."""
    return BASE_SEED + 100 * WORKLOADS[workload] + index


def _mix(z: np.ndarray) -> np.ndarray:
    z = z + GOLDEN
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def raw_u64(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """n consecutive 64-bit outputs of stream ``seed`` starting at element ``offset``."""
    with np.errstate(over="ignore"):
        base = np.uint64(seed % (1 << 64)) * GOLDEN
        idx = np.arange(offset, offset + n, dtype=np.uint64)
        return _mix(base + idx)


def unit(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Uniform doubles in [0, 1) with 53 random bits."""
    return (raw_u64(seed, n, offset) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def integers(shape, seed: int, lo: int = -4, hi: int = 4, dtype=np.float32) -> np.ndarray:
    """Integer values uniform on {lo..hi}, stored as ``dtype``."""
    n = int(np.prod(shape))
    u = unit(seed, n)
    v = np.floor(u * (hi - lo + 1)).astype(np.int64) + lo
    return v.reshape(shape).astype(dtype)


def uniform(shape, seed: int, lo: float = -1.0, hi: float = 1.0, dtype=np.float32) -> np.ndarray:
    n = int(np.prod(shape))
    u = unit(seed, n)
    return (lo + (hi - lo) * u).reshape(shape).astype(dtype)


def normal(shape, seed: int, dtype=np.float32) -> np.ndarray:
    """N(0,1) by Box-Muller from streams ``seed`` and ``seed ^ 0x5bd1e995``."""
    n = int(np.prod(shape))
    u1 = unit(seed, n)
    u2 = unit(seed ^ 0x5BD1E995, n)
    z = np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * np.pi * u2)
    return z.reshape(shape).astype(dtype)


def make(kind: str, shape, seed: int, dtype=np.float32) -> np.ndarray:
    if kind == "int":
        return integers(shape, seed, dtype=dtype)
    if kind == "uniform":
        return uniform(shape, seed, dtype=dtype)
    if kind == "normal":
        return normal(shape, seed, dtype=dtype)
    raise ValueError(f"unknown input kind {kind!r}")


# --------------------------------------------------------------------------
# Device-side twin (torch), for inputs too large to build on the host.
# Integer and uniform families reproduce the numpy bits exactly.
# --------------------------------------------------------------------------

def _torch_mix(z):
    import torch
    def srl(x, s):  # logical right shift on int64 bit patterns
        return (x >> s) & ((1 << (64 - s)) - 1)
    g = torch.tensor(np.int64(np.uint64(GOLDEN).view(np.int64)), dtype=torch.int64, device=z.device)
    m1 = torch.tensor(np.int64(_M1.view(np.int64)), dtype=torch.int64, device=z.device)
    m2 = torch.tensor(np.int64(_M2.view(np.int64)), dtype=torch.int64, device=z.device)
    z = z + g
    z = (z ^ srl(z, 30)) * m1
    z = (z ^ srl(z, 27)) * m2
    return z ^ srl(z, 31)


def torch_unit(seed: int, n: int, device, offset: int = 0, chunk: int = 1 << 26):
    import torch
    out = torch.empty(n, dtype=torch.float64, device=device)
    with np.errstate(over="ignore"):
        base = (np.uint64(seed % (1 << 64)) * GOLDEN).view(np.int64)
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        idx = torch.arange(offset + s, offset + e, dtype=torch.int64, device=device)
        z = _torch_mix(idx + int(base))
        out[s:e] = ((z >> 11) & ((1 << 53) - 1)).to(torch.float64) * (2.0 ** -53)
    return out


def torch_make(kind: str, shape, seed: int, device, dtype=None):
    """Same values as :func:`make` (bit-exact for 'int' and 'uniform'), built on ``device``."""
    import torch
    dtype = dtype or torch.float32
    n = int(np.prod(shape))
    if kind == "int":
        u = torch_unit(seed, n, device)
        v = torch.floor(u * 9.0) - 4.0
    elif kind == "uniform":
        v = -1.0 + 2.0 * torch_unit(seed, n, device)
    elif kind == "normal":
        u1 = torch_unit(seed, n, device)
        u2 = torch_unit(seed ^ 0x5BD1E995, n, device)
        v = torch.sqrt(-2.0 * torch.log1p(-u1)) * torch.cos(2.0 * np.pi * u2)
        del u1, u2
    else:
        raise ValueError(kind)
    return v.to(dtype).reshape(shape)


# --------------------------------------------------------------------------
# Fault-injection draws (positions and magnitudes are inputs to both sides)
# --------------------------------------------------------------------------

def fault_positions(seed: int, n: int, tiles_m: int, tiles_n: int, ksteps: int,
                    m_tb: int, n_tb: int, M: int, N: int, cadence: int,
                    unit_of=None, distinct_units: bool = True):
    """Draw ``n`` fault sites (tile_m, tile_n, kstep, row, col) uniformly.

    Rows/cols are tile-local and always inside the matrix.  With
    ``distinct_units`` two faults never share a (verification unit, period), so
    every fault is correctable under the single-event-upset model (Section 4.1).
    ``unit_of(row, col) -> hashable`` names the verification unit of a
    tile-local element; by default the whole tile is one unit.
    """
    out = []
    used = set()
    stream = 0
    while len(out) < n:
        if stream > 1000 * (n + 1):
            raise RuntimeError("could not place faults without collisions")
        u = unit(seed, 5, offset=5 * stream)
        stream += 1
        tm = int(u[0] * tiles_m)
        tn = int(u[1] * tiles_n)
        ks = int(u[2] * ksteps)
        rows = min(m_tb, M - tm * m_tb)
        cols = min(n_tb, N - tn * n_tb)
        r = int(u[3] * rows)
        c = int(u[4] * cols)
        per = ks // max(1, cadence)
        key = (tm, tn, per, unit_of(r, c) if unit_of else 0)
        if distinct_units and key in used:
            continue
        used.add(key)
        out.append((tm, tn, ks, r, c))
    return out


def log_uniform(seed: int, n: int, lo: float, hi: float) -> np.ndarray:
    u = unit(seed, n)
    return 10.0 ** (np.log10(lo) + u * (np.log10(hi) - np.log10(lo)))


def poisson(seed: int, lam: float, index: int = 0) -> int:
    """Poisson(lam) by inversion of one uniform (Knuth's product method is avoided for large lam)."""
    u = float(unit(seed, 1, offset=index)[0])
    k, p = 0, np.exp(-lam)
    cdf = p
    while u > cdf and k < 10_000:
        k += 1
        p *= lam / k
        cdf += p
    return k


def block(kind: str, seed: int, full_shape, rows, cols, dtype=np.float32) -> np.ndarray:
    """The sub-block [rows[0]:rows[1], cols[0]:cols[1]] of the row-major matrix
    that ``make(kind, full_shape, seed)`` would build, without building it."""
    R, Cn = full_shape
    r0, r1 = rows
    c0, c1 = cols
    out = np.empty((r1 - r0, c1 - c0), dtype=dtype)
    for r in range(r0, r1):
        off = r * Cn + c0
        n = c1 - c0
        if kind == "int":
            u = unit(seed, n, off)
            out[r - r0] = (np.floor(u * 9).astype(np.int64) - 4).astype(dtype)
        elif kind == "uniform":
            out[r - r0] = (-1.0 + 2.0 * unit(seed, n, off)).astype(dtype)
        elif kind == "normal":
            u1 = unit(seed, n, off)
            u2 = unit(seed ^ 0x5BD1E995, n, off)
            out[r - r0] = (np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * np.pi * u2)).astype(dtype)
        else:
            raise ValueError(kind)
    return out
