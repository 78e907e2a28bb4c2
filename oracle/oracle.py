"""Python access to the NaSch oracle (``nasch_oracle.c``).

TEST INFRASTRUCTURE ONLY.  The oracle is the plain serial CPU statement of
the method (the four rules of the handout's model section, the Bernoulli
draw, the ring road, both representations); it exists to check the GPU
library.  Only the tests, the package's smoke check and the benchmark's CPU
baseline leg may import this module.  The library never does.

Two builds of one C source are made with gcc: a serial one and an OpenMP one
(the CPU baseline).  Both give bit-identical results, which is the paper's
reproducibility requirement (assignment item 1: the same seed gives the same
result at any thread count).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "nasch_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LOCK = threading.Lock()
_LIBS: dict[bool, ctypes.CDLL] = {}

TAG_SLOWDOWN = 0
TAG_INIT = 1


class OracleError(RuntimeError):
    pass


def _lib_path(openmp: bool) -> str:
    return os.path.join(_BUILD, "liboracle_omp.so" if openmp else "liboracle.so")


def build(force: bool = False) -> None:
    """Compile both builds of the oracle (gcc, -O2, no target-specific flags)."""
    os.makedirs(_BUILD, exist_ok=True)
    for openmp in (False, True):
        out = _lib_path(openmp)
        if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(_SRC):
            continue
        cmd = ["gcc", "-std=c11", "-O2", "-fPIC", "-shared", "-Wall", "-Wno-unknown-pragmas"]
        if openmp:
            cmd.append("-fopenmp")
        tmp = out + f".tmp{os.getpid()}"
        cmd += [_SRC, "-o", tmp]
        subprocess.run(cmd, check=True)
        os.replace(tmp, out)


def _load(openmp: bool) -> ctypes.CDLL:
    with _LOCK:
        if openmp in _LIBS:
            return _LIBS[openmp]
        build()
        lib = ctypes.CDLL(_lib_path(openmp))
        P = ctypes.c_void_p
        i64, u64, i32, u32 = ctypes.c_int64, ctypes.c_uint64, ctypes.c_int32, ctypes.c_uint32
        lib.oracle_philox4x32_10.argtypes = [P, P, P]
        lib.oracle_philox4x32_10.restype = None
        lib.oracle_philox_many.argtypes = [i64, P, P, P]
        lib.oracle_philox_many.restype = None
        lib.oracle_slow_threshold.argtypes = [ctypes.c_double]
        lib.oracle_slow_threshold.restype = u64
        lib.oracle_floyd_init.argtypes = [i64, i64, u64, u32, P]
        lib.oracle_floyd_init.restype = ctypes.c_int
        lib.oracle_agent_run.argtypes = [i64, i64, i32, u64, u64, u32, u64, i64, P, P, P, P]
        lib.oracle_agent_run.restype = ctypes.c_int
        lib.oracle_grid_run.argtypes = [i64, i32, u64, u64, u32, u64, i64, P, P, P]
        lib.oracle_grid_run.restype = ctypes.c_int
        lib.oracle_open_run.argtypes = [i64, i32, u64, u64, u64, u64, u32, u64, i64, P, P, P]
        lib.oracle_open_run.restype = ctypes.c_int
        lib.oracle_agent_to_grid.argtypes = [i64, i64, P, P, P]
        lib.oracle_agent_to_grid.restype = ctypes.c_int
        lib.oracle_agent_segment.argtypes = [i64, i64, i32, u64, u64, u32, u64, i64, P, P]
        lib.oracle_agent_segment.restype = ctypes.c_int
        lib.oracle_grid_segment.argtypes = [i64, i64, i64, i32, u64, u64, u32, u64, i64, P]
        lib.oracle_grid_segment.restype = ctypes.c_int
        lib.oracle_agent_step_masked.argtypes = [i64, i64, i32, i64, P, P, P, P, P]
        lib.oracle_agent_step_masked.restype = ctypes.c_int
        lib.oracle_set_threads.argtypes = [ctypes.c_int]
        lib.oracle_set_threads.restype = ctypes.c_int
        _LIBS[openmp] = lib
        return lib


def _ptr(a: np.ndarray | None):
    return None if a is None else ctypes.c_void_p(a.ctypes.data)


def _check(status: int, what: str) -> None:
    if status != 0:
        raise OracleError(f"{what} failed with status {status}")


def _key(seed: int) -> np.ndarray:
    return np.array([seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF], dtype=np.uint32)


def philox4x32_10(ctr, seed: int) -> np.ndarray:
    """Philox4x32-10 of one counter (4 words) under key (seed lo, seed hi)."""
    c = np.ascontiguousarray(np.asarray(ctr, dtype=np.uint32).reshape(4))
    out = np.zeros(4, dtype=np.uint32)
    _load(False).oracle_philox4x32_10(_ptr(c), _ptr(_key(seed)), _ptr(out))
    return out


def philox_many(ctrs: np.ndarray, seed: int) -> np.ndarray:
    """Row-wise Philox4x32-10 of an (n, 4) uint32 counter array."""
    c = np.ascontiguousarray(np.asarray(ctrs, dtype=np.uint32).reshape(-1, 4))
    out = np.zeros_like(c)
    _load(False).oracle_philox_many(len(c), _ptr(c), _ptr(_key(seed)), _ptr(out))
    return out


def slow_threshold(p: float) -> int:
    """ceil(p * 2^32): a 32-bit word u means a slowdown iff u < this."""
    return int(_load(False).oracle_slow_threshold(float(p)))


def floyd_init(L: int, N: int, seed: int, road: int = 0) -> np.ndarray:
    """Sorted initial positions: N distinct cells of the ring by Floyd's algorithm."""
    x = np.zeros(max(N, 1), dtype=np.int32)
    _check(_load(False).oracle_floyd_init(L, N, seed, road, _ptr(x)), "floyd_init")
    return x[:N].copy()


def agent_run(L, x, v, vmax, p, seed, road=0, step0=0, T=1, *, openmp=False, thr=None):
    """Run T synchronous steps of the agent form.

    Returns (x, v, sum_v[T], crossings[T]) as new arrays; the inputs are not
    modified.  ``thr`` overrides the threshold computed from ``p``.
    """
    x = np.array(x, dtype=np.int32, copy=True)
    v = np.array(v, dtype=np.uint8, copy=True)
    N = len(x)
    assert len(v) == N
    sv = np.zeros(T, dtype=np.uint64)
    cr = np.zeros(T, dtype=np.uint64)
    t = slow_threshold(p) if thr is None else int(thr)
    st = _load(openmp).oracle_agent_run(L, N, vmax, t, seed, road, step0, T,
                                        _ptr(x), _ptr(v), _ptr(sv), _ptr(cr))
    _check(st, "agent_run")
    return x, v, sv, cr


def agent_step_masked(L, x, v, slow, vmax):
    """One step of the agent form with the rule-3 outcome given per car
    (``slow`` nonzero: the car's Bernoulli trial succeeded) instead of drawn.
    ``x``, ``v``, ``slow``: arrays of shape (count, N), one independent
    state per row, cars in cyclic order.  Returns (x', v') of that shape."""
    x = np.ascontiguousarray(x, dtype=np.int32)
    v = np.ascontiguousarray(v, dtype=np.uint8)
    slow = np.ascontiguousarray(slow, dtype=np.uint8)
    assert x.ndim == 2 and x.shape == v.shape == slow.shape
    count, N = x.shape
    xo = np.zeros_like(x)
    vo = np.zeros_like(v)
    _check(_load(False).oracle_agent_step_masked(L, N, vmax, count, _ptr(x), _ptr(v), _ptr(slow), _ptr(xo),
                                                 _ptr(vo)), "agent_step_masked")
    return xo, vo


def grid_run(cells, vmax, p, seed, road=0, step0=0, T=1, *, openmp=False, thr=None):
    """Run T synchronous steps of the grid form; returns (cells, sum_v, crossings)."""
    c = np.array(cells, dtype=np.int8, copy=True)
    sv = np.zeros(T, dtype=np.uint64)
    cr = np.zeros(T, dtype=np.uint64)
    t = slow_threshold(p) if thr is None else int(thr)
    st = _load(openmp).oracle_grid_run(len(c), vmax, t, seed, road, step0, T,
                                       _ptr(c), _ptr(sv), _ptr(cr))
    _check(st, "grid_run")
    return c, sv, cr


def open_run(cells, vmax, p, alpha, beta, seed, road=0, step0=0, T=1, *, thr=None):
    """Open road (entry before cell 0 with probability alpha, exit after cell
    L-1 open with probability beta; see oracle_open_run): T steps on a copy
    of `cells` (int8, -1 empty).  Returns (cells, sum_v[T], crossings[T])
    with crossings = cars that left."""
    c = np.ascontiguousarray(cells, dtype=np.int8).copy()
    sv = np.zeros(max(T, 1), np.uint64)
    cr = np.zeros(max(T, 1), np.uint64)
    t = slow_threshold(p) if thr is None else thr
    _check(_load(False).oracle_open_run(len(c), vmax, t, slow_threshold(alpha), slow_threshold(beta), seed, road,
                                        step0, T, _ptr(c), _ptr(sv), _ptr(cr)), "oracle_open_run")
    return c, sv[:T], cr[:T]


def agent_to_grid(L, x, v) -> np.ndarray:
    x = np.ascontiguousarray(x, dtype=np.int32)
    v = np.ascontiguousarray(v, dtype=np.uint8)
    cells = np.zeros(L, dtype=np.int8)
    _check(_load(False).oracle_agent_to_grid(L, len(x), _ptr(x), _ptr(v), _ptr(cells)),
           "agent_to_grid")
    return cells


def agent_segment(L, x, v, vmax, p, seed, road=0, step0=0, T=1, *, openmp=False):
    """State of the first len(x)-T of consecutive cars x, v after T steps."""
    x = np.array(x, dtype=np.int32, copy=True)
    v = np.array(v, dtype=np.uint8, copy=True)
    M = len(x)
    st = _load(openmp).oracle_agent_segment(L, M, vmax, slow_threshold(p), seed, road, step0, T,
                                            _ptr(x), _ptr(v))
    _check(st, "agent_segment")
    return x[: M - T].copy(), v[: M - T].copy()


def grid_segment(L, cells, first, vmax, p, seed, road=0, step0=0, T=1):
    """Cells first+T*vmax .. first+W-T*vmax-1 (mod L) after T steps."""
    c = np.array(cells, dtype=np.int8, copy=True)
    W = len(c)
    st = _load(False).oracle_grid_segment(L, W, first, vmax, slow_threshold(p), seed, road,
                                          step0, T, _ptr(c))
    _check(st, "grid_segment")
    m = T * vmax
    return c[m: W - m].copy()


def raster_row(L: int, x: np.ndarray, width: int) -> np.ndarray:
    """One row of the space-time diagram (Fig. 1: the road's cells across,
    time down; darker where cars are) at `width` pixels: pixel i covers the
    cells c with floor(c * width / L) == i and holds floor(255 * cars / cells)
    over them.  x: the cars' cells.  Written from that definition: each car's
    pixel by integer division, each pixel's cell count by counting the cells
    that map to it."""
    L, width = int(L), int(width)
    assert 1 <= width <= L
    x = np.asarray(x, dtype=np.int64)
    cars = np.bincount((x * width) // L, minlength=width)[:width]
    if L <= 1 << 24:
        cells = np.bincount((np.arange(L, dtype=np.int64) * width) // L, minlength=width)
    else:   # the first cell of pixel i is ceil(i * L / width)
        first = (np.arange(width + 1, dtype=object) * L + width - 1) // width
        cells = np.array([int(first[i + 1] - first[i]) for i in range(width)], dtype=np.int64)
    return ((255 * cars) // cells).astype(np.uint8)


def set_threads(n: int) -> int:
    """Set the OpenMP build's thread count; returns the count now in force."""
    return int(_load(True).oracle_set_threads(int(n)))
