"""Python binding of the NaSch C ABI (``include/nasch.h``).

Argument marshalling only: every step of the simulation runs in the CUDA
kernels of ``_build/libnasch.so``.  The library must be built (``build.py``)
and a CUDA device present; nothing here falls back to a CPU path.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

OK = 0
EINVAL = -1
ENOMEM = -2
ECUDA = -3
ETIMEOUT = -4
EBUSY = -5
ECANCELED = -6

LAYOUT_AUTO = 0
LAYOUT_AGENT = 1
LAYOUT_GRID = 2
LAYOUTS = {"auto": LAYOUT_AUTO, "agent": LAYOUT_AGENT, "grid": LAYOUT_GRID}

_STATUS = {EINVAL: "EINVAL", ENOMEM: "ENOMEM", ECUDA: "ECUDA", ETIMEOUT: "ETIMEOUT", EBUSY: "EBUSY",
           ECANCELED: "ECANCELED"}


class NaschError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{_STATUS.get(status, status)}: {message}")
        self.status = status


class Params(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int64), ("N", ctypes.c_int64), ("vmax", ctypes.c_int32),
                ("p", ctypes.c_double), ("seed", ctypes.c_uint64), ("road_id", ctypes.c_uint32),
                ("layout", ctypes.c_int32), ("k", ctypes.c_int32), ("tile", ctypes.c_int32),
                ("stream", ctypes.c_void_p)]


class Info(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int64), ("N", ctypes.c_int64), ("vmax", ctypes.c_int32),
                ("layout", ctypes.c_int32), ("k", ctypes.c_int32), ("tile", ctypes.c_int32),
                ("step", ctypes.c_uint64), ("stats_first", ctypes.c_uint64),
                ("threshold", ctypes.c_uint64), ("ring_kernel", ctypes.c_int32),
                ("blocks", ctypes.c_int32)]


class BatchInfo(ctypes.Structure):
    _fields_ = [("n_roads", ctypes.c_int64), ("super_steps", ctypes.c_int64), ("items", ctypes.c_int64),
                ("device_bytes", ctypes.c_int64), ("vehicle_steps", ctypes.c_int64),
                ("cell_steps", ctypes.c_int64), ("blocks", ctypes.c_int32), ("graphs", ctypes.c_int32),
                ("run_seconds", ctypes.c_double)]


_lib = None
_lock = threading.Lock()


def library_path() -> str:
    """The library this process loads: the debug build when the environment
    sets NASCH_LIBRARY=debug, else the release build."""
    return _build.LIB_DEBUG if os.environ.get("NASCH_LIBRARY") == "debug" else _build.LIB


def load(build_if_missing: bool = False) -> ctypes.CDLL:
    """Load libnasch.so; raises if it is missing (no fallback exists)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = library_path()
        if not os.path.exists(path):
            if not build_if_missing:
                raise RuntimeError(f"{path} is missing: build it with "
                                   "`python -m paper_2309_14311_gb300.build` (needs nvcc)")
            _build.build(debug=path == _build.LIB_DEBUG)
        lib = ctypes.CDLL(path)
        _declare(lib)
        _lib = lib
        return lib


def _declare(lib) -> None:
    P, i64, u64, i32, u32, dbl = (ctypes.c_void_p, ctypes.c_int64, ctypes.c_uint64, ctypes.c_int32,
                                  ctypes.c_uint32, ctypes.c_double)
    H = ctypes.c_void_p
    sig = {
        "nasch_params_init": (None, [P]),
        "nasch_create": (ctypes.c_int, [i64, i64, ctypes.c_int, dbl, u64, P]),
        "nasch_create_ex": (ctypes.c_int, [P, P]),
        "nasch_create_open": (ctypes.c_int, [P, dbl, dbl, P]),
        "nasch_set_state": (ctypes.c_int, [H, P, P, i64, u64]),
        "nasch_run": (ctypes.c_int, [H, i64]),
        "nasch_run_output": (ctypes.c_int, [H, i64, i64, P, i64, P, i32, i64]),
        "nasch_read_state": (ctypes.c_int, [H, P, P, i64]),
        "nasch_read_grid": (ctypes.c_int, [H, P, i64]),
        "nasch_stats": (ctypes.c_int, [H, u64, i64, P, P]),
        "nasch_get_info": (ctypes.c_int, [H, P]),
        "nasch_synchronize": (ctypes.c_int, [H]),
        "nasch_destroy": (None, [H]),
        "nasch_last_error": (ctypes.c_char_p, []),
        "nasch_slow_threshold": (u64, [dbl]),
        "nasch_floyd_init": (ctypes.c_int, [i64, i64, u64, u32, P]),
        "nasch_philox_device": (ctypes.c_int, [i64, P, u64, P]),
        "nasch_calibrate_philox": (ctypes.c_int, [i64, P, P]),
        "nasch_submit": (ctypes.c_int, [P, i64, P, P]),
        "nasch_batch_wait": (ctypes.c_int, [H, i64]),
        "nasch_batch_cancel": (ctypes.c_int, [H]),
        "nasch_batch_read_state": (ctypes.c_int, [H, i64, P, P, i64]),
        "nasch_batch_read_grid": (ctypes.c_int, [H, i64, P, i64]),
        "nasch_batch_stats": (ctypes.c_int, [H, i64, u64, i64, P, P]),
        "nasch_batch_stats_sum": (ctypes.c_int, [H, i64, u64, i64, P, P]),
        "nasch_batch_get_info": (ctypes.c_int, [H, P]),
        "nasch_batch_road_layout": (ctypes.c_int, [H, i64, P]),
        "nasch_batch_destroy": (None, [H]),
        "nasch_set_tuning": (ctypes.c_int, [dbl, i32, i32]),
        "nasch_server_poll_series": (ctypes.c_int, [H, P, i64, P, P, i64, P]),
        "nasch_set_tuning_table": (ctypes.c_int, [P, i64]),
        "nasch_get_tuning_table": (ctypes.c_int, [P, i64, P]),
        "nasch_tuned_choice": (ctypes.c_int, [P, P, P, P]),
        "nasch_segment_run": (ctypes.c_int, [P, P, i64, i32, i64, i64, i32, dbl, u64, u32, u64, i32, P, P, P]),
        "nasch_floyd_init_device_noalloc": (ctypes.c_int, [i64, i64, u64, u32, P, P]),
        "nasch_selftest_bounded_wait": (ctypes.c_int, [i64, P]),
        "nasch_server_config_init": (None, [P]),
        "nasch_server_create": (ctypes.c_int, [P, P]),
        "nasch_server_submit": (ctypes.c_int, [H, P, i64, u64]),
        "nasch_server_step": (ctypes.c_int, [H, P]),
        "nasch_server_drain": (ctypes.c_int, [H, i64]),
        "nasch_server_poll": (ctypes.c_int, [H, P, i64, P]),
        "nasch_server_result": (ctypes.c_int, [H, u64, P, P, i64, P, P, i64]),
        "nasch_server_release": (ctypes.c_int, [H, u64]),
        "nasch_server_cancel": (ctypes.c_int, [H, u64]),
        "nasch_server_get_info": (ctypes.c_int, [H, P]),
        "nasch_server_destroy": (None, [H]),
        "nasch_get_tuning": (ctypes.c_int, [P, P, P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args


def _check(status: int) -> None:
    if status != OK:
        msg = load().nasch_last_error()
        raise NaschError(status, msg.decode() if msg else "")


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


def slow_threshold(p: float) -> int:
    return int(load().nasch_slow_threshold(float(p)))


def floyd_init(L: int, N: int, seed: int, road: int = 0) -> np.ndarray:
    x = np.zeros(max(N, 1), dtype=np.int32)
    _check(load().nasch_floyd_init(L, N, seed, road, _ptr(x)))
    return x[:N].copy()


def philox_device(ctr: np.ndarray, seed: int) -> np.ndarray:
    c = np.ascontiguousarray(np.asarray(ctr, dtype=np.uint32).reshape(-1, 4))
    out = np.zeros_like(c)
    _check(load().nasch_philox_device(len(c), _ptr(c), seed, _ptr(out)))
    return out


def floyd_init_device_noalloc(L: int, N: int, seed: int, road: int, x_dev_ptr: int, stream=None) -> None:
    """Floyd start positions written to a caller-owned device buffer (int32,
    N entries) without any device allocation by the library; asynchronous on
    `stream`.  Roads of at most 2^24 cells."""
    _check(load().nasch_floyd_init_device_noalloc(int(L), int(N), int(seed), int(road), ctypes.c_void_p(x_dev_ptr),
                                                  _stream_handle(stream)))


def segment_run(in_ptr: int, out_ptr: int, owned: int, halo: int, first_cell: int, L: int, vmax: int, p: float,
                seed: int, road_id: int, step0: int, k: int, sum_v_ptr: int, crossings_ptr: int, stream=None) -> None:
    """nasch_segment_run on caller-owned device buffers (raw pointers)."""
    _check(load().nasch_segment_run(ctypes.c_void_p(in_ptr), ctypes.c_void_p(out_ptr), int(owned), int(halo),
                                    int(first_cell), int(L), int(vmax), float(p), int(seed), int(road_id),
                                    int(step0), int(k), ctypes.c_void_p(sum_v_ptr), ctypes.c_void_p(crossings_ptr),
                                    _stream_handle(stream)))


def selftest_bounded_wait(limit_ms: int = 50):
    """Run the bounded-wait self-test kernel; returns (status code, status word)."""
    w = ctypes.c_uint32()
    st = load().nasch_selftest_bounded_wait(int(limit_ms), ctypes.byref(w))
    return st, w.value


def calibrate_philox(draws_per_thread: int = 1 << 14) -> float:
    """Draws per second of the bare rule-3 Philox draw on this GPU."""
    rate = ctypes.c_double()
    secs = ctypes.c_double()
    _check(load().nasch_calibrate_philox(draws_per_thread, ctypes.byref(rate), ctypes.byref(secs)))
    return rate.value


class Road:
    """One road with device-resident state (a ``nasch_handle``): a ring, or
    with ``open=(alpha, beta)`` an open road (entry before cell 0 with
    probability alpha, exit after cell L-1 open with probability beta; grid
    layout, one step per launch)."""

    def __init__(self, L: int, N: int, vmax: int = 5, p: float = 0.0, seed: int = 0, road_id: int = 0,
                 layout: str | int = "auto", k: int = 0, tile: int = 0, stream=None,
                 open: tuple[float, float] | None = None):
        lib = load()
        prm = Params()
        lib.nasch_params_init(ctypes.byref(prm))
        prm.L, prm.N, prm.vmax, prm.p, prm.seed, prm.road_id = L, N, vmax, float(p), seed, road_id
        prm.layout = LAYOUTS[layout] if isinstance(layout, str) else int(layout)
        prm.k, prm.tile = k, tile
        prm.stream = _stream_handle(stream)
        self._stream_ref = stream
        h = ctypes.c_void_p()
        if open is None:
            _check(lib.nasch_create_ex(ctypes.byref(prm), ctypes.byref(h)))
        else:
            _check(lib.nasch_create_open(ctypes.byref(prm), float(open[0]), float(open[1]), ctypes.byref(h)))
        self._h = h
        self.L, self.N, self.vmax, self.p, self.seed, self.road_id = L, N, vmax, p, seed, road_id

    def close(self) -> None:
        if getattr(self, "_h", None):
            load().nasch_destroy(self._h)
            self._h = None

    __del__ = close

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def handle(self):
        return self._h

    def info(self) -> Info:
        inf = Info()
        _check(load().nasch_get_info(self._h, ctypes.byref(inf)))
        return inf

    @property
    def step(self) -> int:
        return int(self.info().step)

    def set_state(self, x, v, step: int = 0) -> None:
        x = np.ascontiguousarray(x, dtype=np.int32)
        v = np.ascontiguousarray(v, dtype=np.uint8)
        _check(load().nasch_set_state(self._h, _ptr(x), _ptr(v), len(x), step))

    def run(self, steps: int) -> None:
        _check(load().nasch_run(self._h, steps))

    def run_output(self, steps: int, per: int, snapshots: np.ndarray | None = None,
                   raster: np.ndarray | None = None) -> None:
        """Run `steps` steps with output after every `per` steps: snapshot j
        of the cells into snapshots[j % len(snapshots)] (shape (n, L), int8)
        and raster row j into raster[j % len(raster)] (shape (n, width),
        uint8).  Either may be None.  Synchronous."""
        sp, sn, rp, rw, rn = None, 0, None, 0, 0
        if snapshots is not None:
            assert snapshots.dtype == np.int8 and snapshots.ndim == 2 and snapshots.shape[1] == self.L
            assert snapshots.flags.c_contiguous
            sp, sn = _ptr(snapshots), snapshots.shape[0]
        if raster is not None:
            assert raster.dtype == np.uint8 and raster.ndim == 2 and raster.flags.c_contiguous
            rp, rw, rn = _ptr(raster), raster.shape[1], raster.shape[0]
        _check(load().nasch_run_output(self._h, steps, per, sp, sn, rp, rw, rn))

    def synchronize(self) -> None:
        _check(load().nasch_synchronize(self._h))

    def read_state(self, out_x: np.ndarray | None = None, out_v: np.ndarray | None = None):
        x = out_x if out_x is not None else np.empty(max(self.N, 1), dtype=np.int32)
        v = out_v if out_v is not None else np.empty(max(self.N, 1), dtype=np.uint8)
        _check(load().nasch_read_state(self._h, _ptr(x), _ptr(v), min(len(x), len(v))))
        return x[: self.N], v[: self.N]

    def read_grid(self) -> np.ndarray:
        c = np.empty(self.L, dtype=np.int8)
        _check(load().nasch_read_grid(self._h, _ptr(c), self.L))
        return c

    def stats(self, first_step: int | None = None, count: int | None = None):
        inf = self.info()
        first = int(inf.stats_first) if first_step is None else first_step
        n = int(inf.step) - first if count is None else count
        sv = np.zeros(max(n, 1), dtype=np.uint64)
        cr = np.zeros(max(n, 1), dtype=np.uint64)
        _check(load().nasch_stats(self._h, first, n, _ptr(sv), _ptr(cr)))
        return sv[:n], cr[:n]


def _stream_handle(stream):
    """cudaStream_t of a torch.cuda.Stream (or a raw integer handle), else None."""
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


def set_tuning(rho_star: float, k_agent: int = 0, k_grid: int = 0) -> None:
    """Density below which AUTO picks the agent layout, and default fusion depths."""
    _check(load().nasch_set_tuning(float(rho_star), int(k_agent), int(k_grid)))


def get_tuning():
    r, ka, kg = ctypes.c_double(), ctypes.c_int32(), ctypes.c_int32()
    _check(load().nasch_get_tuning(ctypes.byref(r), ctypes.byref(ka), ctypes.byref(kg)))
    return r.value, ka.value, kg.value


def set_tuning_table(entries: list[dict]) -> None:
    """Per-road tuning (nasch_set_tuning_table): dicts with the fields of
    TuningEntry; layout may be given as "auto", "agent" or "grid"."""
    arr = (TuningEntry * max(len(entries), 1))()
    for i, e in enumerate(entries):
        for f in TUNING_FIELDS:
            v = e.get(f, 0)
            if f == "layout" and isinstance(v, str):
                v = LAYOUTS[v]
            setattr(arr[i], f, v)
    _check(load().nasch_set_tuning_table(arr, len(entries)))


def get_tuning_table() -> list[dict]:
    n = ctypes.c_int64()
    _check(load().nasch_get_tuning_table(None, 0, ctypes.byref(n)))
    arr = (TuningEntry * max(n.value, 1))()
    _check(load().nasch_get_tuning_table(arr, n.value, ctypes.byref(n)))
    return [{f: getattr(arr[i], f) for f in TUNING_FIELDS} for i in range(n.value)]


def tuned_choice(road: dict) -> tuple[int, int, int]:
    """(layout, k, tile) a batch would give this road (nasch_tuned_choice)."""
    prm = make_params(**road)
    lay, k, tile = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    _check(load().nasch_tuned_choice(ctypes.byref(prm), ctypes.byref(lay), ctypes.byref(k), ctypes.byref(tile)))
    return lay.value, k.value, tile.value


def make_params(L, N, vmax=5, p=0.0, seed=0, road_id=0, layout="auto", k=0, tile=0, stream=None) -> Params:
    prm = Params()
    load().nasch_params_init(ctypes.byref(prm))
    prm.L, prm.N, prm.vmax, prm.p, prm.seed, prm.road_id = int(L), int(N), int(vmax), float(p), int(seed), int(road_id)
    prm.layout = LAYOUTS[layout] if isinstance(layout, str) else int(layout)
    prm.k, prm.tile = int(k), int(tile)
    prm.stream = _stream_handle(stream)
    return prm


class Batch:
    """Many roads run together (``nasch_submit``).  ``roads`` are dicts with
    the keys of ``make_params``; ``steps[i]`` steps are run on road i."""

    def __init__(self, roads, steps, stream=None):
        lib = load()
        n = len(roads)
        arr = (Params * n)()
        for i, r in enumerate(roads):
            arr[i] = make_params(**r, stream=stream if i == 0 else None)
        st = np.ascontiguousarray(np.asarray(steps, dtype=np.int64))
        assert len(st) == n
        self._stream_ref = stream
        self._roads = [dict(r) for r in roads]
        self._steps = st.copy()
        h = ctypes.c_void_p()
        _check(lib.nasch_submit(arr, n, _ptr(st), ctypes.byref(h)))
        self._h = h
        self.n = n

    def close(self) -> None:
        if getattr(self, "_h", None):
            load().nasch_batch_destroy(self._h)
            self._h = None

    __del__ = close

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def wait(self, timeout_ms: int = -1) -> None:
        _check(load().nasch_batch_wait(self._h, int(timeout_ms)))

    def cancel(self) -> None:
        _check(load().nasch_batch_cancel(self._h))

    def info(self) -> BatchInfo:
        inf = BatchInfo()
        _check(load().nasch_batch_get_info(self._h, ctypes.byref(inf)))
        return inf

    def layout(self, i: int) -> int:
        lay = ctypes.c_int32()
        _check(load().nasch_batch_road_layout(self._h, i, ctypes.byref(lay)))
        return lay.value

    def read_state(self, i: int):
        N = int(self._roads[i]["N"])
        x = np.empty(max(N, 1), dtype=np.int32)
        v = np.empty(max(N, 1), dtype=np.uint8)
        _check(load().nasch_batch_read_state(self._h, i, _ptr(x), _ptr(v), len(x)))
        return x[:N], v[:N]

    def read_grid(self, i: int) -> np.ndarray:
        L = int(self._roads[i]["L"])
        c = np.empty(L, dtype=np.int8)
        _check(load().nasch_batch_read_grid(self._h, i, _ptr(c), L))
        return c

    def stats(self, i: int, first: int = 0, count: int | None = None):
        n = int(self._steps[i]) - first if count is None else count
        sv = np.zeros(max(n, 1), dtype=np.uint64)
        cr = np.zeros(max(n, 1), dtype=np.uint64)
        _check(load().nasch_batch_stats(self._h, i, first, n, _ptr(sv), _ptr(cr)))
        return sv[:n], cr[:n]

    def stats_sum(self, i: int, first: int, count: int):
        a, c = ctypes.c_uint64(), ctypes.c_uint64()
        _check(load().nasch_batch_stats_sum(self._h, i, first, count, ctypes.byref(a), ctypes.byref(c)))
        return a.value, c.value


class ServerConfig(ctypes.Structure):
    _fields_ = [("memory_budget", ctypes.c_int64), ("steps_per_tick", ctypes.c_int32),
                ("max_resident", ctypes.c_int32), ("keep_state", ctypes.c_int32), ("stream", ctypes.c_void_p),
                ("max_steps_per_tick", ctypes.c_int32), ("ticks_in_flight", ctypes.c_int32),
                ("target_tick_ms", ctypes.c_double)]


class RequestResult(ctypes.Structure):
    _fields_ = [("request_id", ctypes.c_uint64), ("status", ctypes.c_int32), ("layout", ctypes.c_int32),
                ("steps", ctypes.c_int64), ("vehicles", ctypes.c_int64), ("submit_time", ctypes.c_double),
                ("admit_time", ctypes.c_double), ("done_time", ctypes.c_double)]


class ServerInfo(ctypes.Structure):
    _fields_ = [("queued", ctypes.c_int64), ("resident", ctypes.c_int64), ("completed", ctypes.c_int64),
                ("bytes_in_use", ctypes.c_int64), ("ticks", ctypes.c_int64), ("vehicle_steps_done", ctypes.c_int64),
                ("blocks", ctypes.c_int32), ("now", ctypes.c_double), ("gpu_busy_seconds", ctypes.c_double),
                ("last_tick_super_steps", ctypes.c_int32), ("pad", ctypes.c_int32)]


class TuningEntry(ctypes.Structure):
    _fields_ = [("L_min", ctypes.c_int64), ("L_max", ctypes.c_int64), ("rho_min", ctypes.c_double),
                ("rho_max", ctypes.c_double), ("vmax_min", ctypes.c_int32), ("vmax_max", ctypes.c_int32),
                ("draw", ctypes.c_int32), ("layout", ctypes.c_int32), ("k", ctypes.c_int32), ("tile", ctypes.c_int32)]


TUNING_FIELDS = [f for f, _ in TuningEntry._fields_]


class SeriesChunk(ctypes.Structure):
    _fields_ = [("request_id", ctypes.c_uint64), ("first_step", ctypes.c_int64), ("count", ctypes.c_int64),
                ("offset", ctypes.c_int64)]


class Server:
    """Continuous-batching request loop (``nasch_server_*``)."""

    def __init__(self, memory_budget: int = 40 << 30, steps_per_tick: int = 8, max_resident: int = 4096,
                 keep_state: bool = False, stream=None, max_steps_per_tick: int | None = None,
                 ticks_in_flight: int | None = None, target_tick_ms: float | None = None):
        lib = load()
        cfg = ServerConfig()
        lib.nasch_server_config_init(ctypes.byref(cfg))
        cfg.memory_budget, cfg.steps_per_tick, cfg.max_resident = int(memory_budget), int(steps_per_tick), int(max_resident)
        if max_steps_per_tick is not None:
            cfg.max_steps_per_tick = int(max_steps_per_tick)
        if ticks_in_flight is not None:
            cfg.ticks_in_flight = int(ticks_in_flight)
        if target_tick_ms is not None:
            cfg.target_tick_ms = float(target_tick_ms)
        cfg.keep_state = 1 if keep_state else 0
        cfg.stream = _stream_handle(stream)
        self._stream_ref = stream
        h = ctypes.c_void_p()
        _check(lib.nasch_server_create(ctypes.byref(cfg), ctypes.byref(h)))
        self._h = h
        self._roads = {}

    def close(self) -> None:
        if getattr(self, "_h", None):
            load().nasch_server_destroy(self._h)
            self._h = None

    __del__ = close

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def submit(self, road: dict, steps: int, request_id: int) -> None:
        prm = make_params(**road)
        _check(load().nasch_server_submit(self._h, ctypes.byref(prm), int(steps), int(request_id)))
        self._roads[int(request_id)] = (int(road["N"]), int(steps))

    def step(self) -> int:
        pending = ctypes.c_int64()
        _check(load().nasch_server_step(self._h, ctypes.byref(pending)))
        return pending.value

    def drain(self, timeout_ms: int = -1) -> None:
        _check(load().nasch_server_drain(self._h, int(timeout_ms)))

    def poll(self, cap: int = 4096):
        out = (RequestResult * cap)()
        n = ctypes.c_int64()
        _check(load().nasch_server_poll(self._h, out, cap, ctypes.byref(n)))
        return [dict(request_id=r.request_id, status=r.status, layout=r.layout, steps=r.steps, vehicles=r.vehicles,
                     submit_time=r.submit_time, admit_time=r.admit_time, done_time=r.done_time)
                for r in out[: n.value]]

    def result(self, request_id: int, with_state: bool = False):
        N, T = self._roads[int(request_id)]
        sv = np.zeros(max(T, 1), dtype=np.uint64)
        cr = np.zeros(max(T, 1), dtype=np.uint64)
        if with_state:
            x = np.zeros(max(N, 1), dtype=np.int32)
            v = np.zeros(max(N, 1), dtype=np.uint8)
            _check(load().nasch_server_result(self._h, int(request_id), _ptr(sv), _ptr(cr), len(sv), _ptr(x), _ptr(v),
                                              len(x)))
            return sv[:T], cr[:T], x[:N], v[:N]
        _check(load().nasch_server_result(self._h, int(request_id), _ptr(sv), _ptr(cr), len(sv), None, None, 0))
        return sv[:T], cr[:T]

    def poll_series(self, cap_chunks: int = 4096, cap_steps: int = 1 << 20):
        """Newly finished steps of admitted requests: a list of
        (request_id, first_step, sum_v, crossings) with array copies."""
        buf = getattr(self, "_series_buf", None)
        if buf is None or len(buf[0]) < cap_chunks or len(buf[1]) < max(cap_steps, 1):
            buf = ((SeriesChunk * cap_chunks)(), np.zeros(max(cap_steps, 1), dtype=np.uint64),
                   np.zeros(max(cap_steps, 1), dtype=np.uint64))
            self._series_buf = buf
        chunks, sv, cr = buf
        n = ctypes.c_int64()
        _check(load().nasch_server_poll_series(self._h, chunks, cap_chunks, _ptr(sv), _ptr(cr), cap_steps,
                                               ctypes.byref(n)))
        return [(c.request_id, c.first_step, sv[c.offset:c.offset + c.count].copy(),
                 cr[c.offset:c.offset + c.count].copy()) for c in chunks[: n.value]]

    def release(self, request_id: int) -> None:
        _check(load().nasch_server_release(self._h, int(request_id)))
        self._roads.pop(int(request_id), None)

    def cancel(self, request_id: int) -> None:
        _check(load().nasch_server_cancel(self._h, int(request_id)))

    def info(self) -> ServerInfo:
        inf = ServerInfo()
        _check(load().nasch_server_get_info(self._h, ctypes.byref(inf)))
        return inf
