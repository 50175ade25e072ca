"""Continuous-batching server for CBCT reconstruction requests (CGLS).

Requests (geometry, angles, projections, iteration count) arrive over time.
The scheduler keeps up to `max_slots` reconstructions resident on the GPU at
once, each with its own stream, geometry handle and CGLS state (iterates stay
in HBM from admission to completion).  A request is admitted, in arrival
order, as soon as a slot is free and its HBM footprint fits the remaining
budget; it does not wait for the requests already running to finish.  Every
scheduler tick enqueues the next iterations of every resident request on its
stream (as replays of a captured CUDA graph of two CGLS iterations), so
different requests' projections and backprojections overlap on the device.
Finished requests are detected with events, copied back, and their slot and
memory returned to the pool.

`run_plain` is the one-at-a-time reference path: each request is solved
alone with tigre_cgls, in arrival order.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field

import numpy as np
import torch

from . import tigre


@dataclass
class Request:
    rid: int
    geo: dict
    angles: np.ndarray
    proj: torch.Tensor            # host (pinned preferred) projections, F32, BF16 or F16:
                                  # the reconstruction stores its iterates in this type
    n_iter: int = 15
    arrival: float = 0.0          # seconds after the start of the run


@dataclass
class Result:
    rid: int
    x: torch.Tensor               # host F32 volume (widened from the storage type)
    resid: np.ndarray
    arrival: float
    admitted: float
    finished: float

    @property
    def latency(self) -> float:
        return self.finished - self.arrival


def footprint_bytes(geo: dict, n_angles: int, elem: int = 4) -> int:
    """HBM needed by one resident CGLS reconstruction stored in elem-byte
    values: x, p, s (volume-sized), b, r, q (projection-sized), the forward
    projector's two padded layouts and their quad copies (5 padded volumes
    each), the backprojector's padded projections, plus 64 MiB of slack."""
    nx, ny, nz = geo["n_voxel"]
    nu, nv = geo["n_det"]
    vol = elem * nx * ny * nz
    padded = elem * (nx + 4) * (ny + 4) * (nz + 4)
    proj = elem * nu * nv * n_angles
    return 3 * vol + 4 * proj + 10 * padded + (64 << 20)


_STORAGE = (torch.float32, torch.bfloat16, torch.float16)


def storage_dtype(req: Request) -> torch.dtype:
    return req.proj.dtype if req.proj.dtype in _STORAGE else torch.float32


def request_bytes(req: Request) -> int:
    return footprint_bytes(req.geo, len(req.angles), storage_dtype(req).itemsize)


def work_estimate(req: Request) -> float:
    """Voxel-angle pairs visited by the whole reconstruction."""
    return float(np.prod(req.geo["n_voxel"])) * len(req.angles) * (req.n_iter + 1)


def admit(queue: list[Request], n_active: int, used: int, max_slots: int, budget: int,
          policy: str = "fifo") -> list[Request]:
    """Take from `queue` (in place) the requests to admit now, in order: while
    a slot is free and the next request's footprint fits the HBM left (a
    request that fits nothing is admitted alone, when nothing else is
    resident).  fifo keeps arrival order (a large request at the head waits
    and holds the ones behind it); sjf first sorts the queue by estimated
    work."""
    if policy == "sjf":
        queue.sort(key=lambda r: (work_estimate(r), r.arrival, r.rid))
    out: list[Request] = []
    while queue and n_active + len(out) < max_slots:
        need = request_bytes(queue[0])
        if used + need > budget and n_active + len(out) > 0:
            break
        out.append(queue.pop(0))
        used += need
    return out


@dataclass
class _Slot:
    req: Request
    G: tigre.Geometry
    stream: torch.cuda.Stream
    b: torch.Tensor
    x: torch.Tensor
    state: object
    issued: int
    admitted: float
    done_event: torch.cuda.Event = field(default_factory=lambda: torch.cuda.Event())
    bytes: int = 0


class Server:
    def __init__(self, max_slots: int = 8, hbm_budget: int | None = None, graph: bool = True,
                 iters_per_tick: int = 2, device: int = 0, policy: str = "fifo"):
        """policy: "fifo" admits in arrival order; "sjf" admits the queued
        request with the least estimated work (voxels x angles x iterations)
        first, which shortens the typical latency when big and small
        reconstructions are mixed."""
        if policy not in ("fifo", "sjf"):
            raise ValueError("policy must be 'fifo' or 'sjf'")
        self.policy = policy
        self.max_slots = max_slots
        self.graph = graph
        self.iters_per_tick = max(1, iters_per_tick)
        self.device = torch.device("cuda", device)
        if hbm_budget is None:
            free, _ = torch.cuda.mem_get_info(self.device)
            hbm_budget = int(0.8 * free)
        self.hbm_budget = hbm_budget

    def _admit(self, req: Request, now: float) -> _Slot:
        stream = torch.cuda.Stream(device=self.device)
        with torch.cuda.stream(stream):
            G = tigre.Geometry(req.geo, req.angles)
            dt = storage_dtype(req)
            b = req.proj.to(self.device, dtype=dt, non_blocking=True)
            x = torch.empty(G.vol_shape, device=self.device, dtype=dt)  # zeroed by the library
            state = tigre.tigre_cgls_begin(G.handle, b, x, n_iter_hint=req.n_iter,
                                           stream=stream, graph=self.graph, x0_zero=True)
        return _Slot(req, G, stream, b, x, state, 0, now, bytes=request_bytes(req))

    def _finish(self, s: _Slot, now: float) -> Result:
        resid = tigre.tigre_cgls_history(s.state, s.req.n_iter)  # syncs the slot's stream
        x = s.x.float().cpu()
        tigre.tigre_cgls_end(s.state)
        s.G.close()
        return Result(s.req.rid, x, resid, s.req.arrival, s.admitted, now)

    def run(self, requests: list[Request], realtime: bool = True) -> list[Result]:
        """Serve requests (arrival offsets in seconds) and return results in
        completion order."""
        pending = sorted(requests, key=lambda r: (r.arrival, r.rid))
        queue: list[Request] = []
        active: list[_Slot] = []
        results: list[Result] = []
        used = 0
        t0 = time.perf_counter()
        while pending or queue or active:
            now = time.perf_counter() - t0
            while pending and (pending[0].arrival <= now or not realtime):
                queue.append(pending.pop(0))
            # Admission as slots and memory free up (arrival order, or least
            # work first).
            for req in admit(queue, len(active), used, self.max_slots, self.hbm_budget,
                             self.policy):
                slot = self._admit(req, time.perf_counter() - t0)
                used += slot.bytes
                active.append(slot)
            # One tick of work for every resident reconstruction.
            for s in active:
                if s.issued < s.req.n_iter:
                    n = min(self.iters_per_tick, s.req.n_iter - s.issued)
                    with torch.cuda.stream(s.stream):
                        tigre.tigre_cgls_iterate(s.state, n)
                    s.issued += n
                    if s.issued == s.req.n_iter:
                        s.done_event.record(s.stream)
            # Retire finished reconstructions.
            still = []
            for s in active:
                if s.issued == s.req.n_iter and s.done_event.query():
                    results.append(self._finish(s, time.perf_counter() - t0))
                    used -= s.bytes
                else:
                    still.append(s)
            active = still
            if not active and not queue and pending and realtime:
                time.sleep(max(0.0, pending[0].arrival - (time.perf_counter() - t0)))
            elif active and all(s.issued == s.req.n_iter for s in active):
                time.sleep(0.0005)
        return results


def run_plain(requests: list[Request], realtime: bool = True,
              device: int = 0) -> list[Result]:
    """One request at a time, arrival order, each solved alone by tigre_cgls."""
    dev = torch.device("cuda", device)
    results = []
    t0 = time.perf_counter()
    for req in sorted(requests, key=lambda r: (r.arrival, r.rid)):
        now = time.perf_counter() - t0
        if realtime and req.arrival > now:
            time.sleep(req.arrival - now)
        admitted = time.perf_counter() - t0
        with tigre.Geometry(req.geo, req.angles) as G:
            dt = storage_dtype(req)
            b = req.proj.to(dev, dtype=dt)
            x = torch.empty(G.vol_shape, device=dev, dtype=dt)  # zeroed by the library
            resid = tigre.tigre_cgls(G.handle, b, x, req.n_iter, x0_zero=True)
            xh = x.float().cpu()
        results.append(Result(req.rid, xh, resid, req.arrival, admitted,
                              time.perf_counter() - t0))
    return results


def latency_stats(results: list[Result]) -> dict:
    lat = np.array([r.latency for r in results])
    span = max(r.finished for r in results) - min(r.arrival for r in results)
    return {"p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "mean_s": float(lat.mean()), "makespan_s": float(span),
            "throughput_req_s": len(results) / span}


def poisson_requests(n: int, rate: float, seed: int, make) -> list[Request]:
    """n requests with exponential inter-arrival times (rate per second);
    make(i, rng) returns (geo, angles, proj, n_iter)."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for i in range(n):
        t += rng.exponential(1.0 / rate)
        geo, ang, proj, n_iter = make(i, rng)
        out.append(Request(i, geo, ang, proj, n_iter, t))
    return out
