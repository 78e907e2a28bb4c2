"""Serving driver: a Poisson stream of simulation requests against the
continuous-batching server (``nasch_server_*``), with latency statistics.

Requests arrive at scheduled times (unit-rate arrival times divided by the
offered rate); each is submitted when its time comes, and the loop keeps
scheduling rounds going (admission by memory budget, one tick of launches
over all resident roads per round).  Latency is a request's completion time
(when the host saw its last launch finish) minus its scheduled arrival.
"""
from __future__ import annotations

import time

import numpy as np

from . import nasch as NS
from . import workloads as WL


def run_poisson(requests: list[dict], rate: float, memory_budget: int = 40 << 30, steps_per_tick: int = 8,
                max_resident: int = 4096, stream=None, time_limit_s: float | None = None, keep_state: bool = False,
                on_result=None, max_steps_per_tick: int | None = None, ticks_in_flight: int | None = None,
                target_tick_ms: float | None = None, stream_series: bool = False):
    """Serve `requests` (rows of the request table: road keys, T, arrival at
    unit rate) arriving at `rate` requests per second (rate = inf: all at
    once).  Returns a summary: latency percentiles, aggregate
    vehicle-updates/s, the GPU's busy fraction, and counts.  With
    `stream_series` the per-step series are streamed back while requests
    run (nasch_server_poll_series) and the steps received are counted."""
    n = len(requests)
    arrivals = np.array([r["arrival"] for r in requests], dtype=np.float64)
    arrivals = np.zeros_like(arrivals) if rate == float("inf") else arrivals / rate
    done = {}
    streamed_steps = 0
    with NS.Server(memory_budget=memory_budget, steps_per_tick=steps_per_tick, max_resident=max_resident,
                   keep_state=keep_state, stream=stream, max_steps_per_tick=max_steps_per_tick,
                   ticks_in_flight=ticks_in_flight, target_tick_ms=target_tick_ms) as srv:
        offset = srv.info().now - time.perf_counter()
        t_start = time.perf_counter()
        origin = t_start + offset - arrivals[0] if n else 0.0   # server clock of arrival time 0
        i = 0
        while len(done) < n:
            now = time.perf_counter() - t_start + arrivals[0]
            while i < n and arrivals[i] <= now:
                r = requests[i]
                srv.submit(WL.road_params(r), r["T"], i)
                i += 1
            pending = srv.step()
            if stream_series:
                streamed_steps += sum(len(c[2]) for c in srv.poll_series())
            for res in srv.poll():
                done[res["request_id"]] = res
                if on_result is not None:
                    on_result(srv, res)
                if stream_series:
                    streamed_steps += sum(len(c[2]) for c in srv.poll_series())
                srv.release(res["request_id"])
            if pending == 0 and i < n:
                wait = arrivals[i] - (time.perf_counter() - t_start + arrivals[0])
                if wait > 0:
                    time.sleep(min(wait, 0.01))
            if time_limit_s is not None and time.perf_counter() - t_start > time_limit_s:
                break
        info = srv.info()
    ids = sorted(done)
    lat = np.array([done[k]["done_time"] - (origin + arrivals[k]) for k in ids])
    queue_wait = np.array([done[k]["admit_time"] - (origin + arrivals[k]) for k in ids])
    veh = sum(requests[k]["N"] * requests[k]["T"] for k in ids if done[k]["status"] == NS.OK)
    span = (max(done[k]["done_time"] for k in ids) - origin - arrivals[0]) if ids else 0.0
    return {
        "requests": n, "completed": len(ids), "rate_per_s": rate,
        "latency_p50_s": float(np.percentile(lat, 50)) if len(lat) else None,
        "latency_p99_s": float(np.percentile(lat, 99)) if len(lat) else None,
        "latency_mean_s": float(lat.mean()) if len(lat) else None,
        "queue_wait_p50_s": float(np.percentile(queue_wait, 50)) if len(lat) else None,
        "vehicle_updates": int(veh),
        "vehicle_updates_per_s": veh / span if span > 0 else None,
        "span_s": span, "ticks": int(info.ticks),
        "gpu_busy_s": info.gpu_busy_seconds, "gpu_busy_fraction": info.gpu_busy_seconds / span if span > 0 else None,
        "streamed_steps": streamed_steps if stream_series else None,
    }
