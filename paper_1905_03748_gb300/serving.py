"""Continuous-batching server for CBCT reconstruction requests (CGLS).

Requests (geometry, angles, projections, iteration count) arrive over time.
The scheduler keeps up to `max_slots` reconstructions resident on the GPU at
once (iterates stay in HBM from admission to completion).  A request is
admitted, in arrival order, as soon as a slot is free and its HBM footprint
fits the remaining budget; it does not wait for the requests already running
to finish.  Requests queued behind it with the same geometry, angles,
storage type and iteration count join it, up to `max_batch`: the group runs
as one batched CGLS (tigre_cgls_batch_*), whose every iteration projects the
whole group in one forward launch and backprojects it in one backprojection
launch, captured with the group's vector updates in one CUDA graph of two
iterations.  Each group has its own stream and geometry handle; every
scheduler tick enqueues the next iterations of every resident group, so
different groups' launches overlap on the device.  Finished groups are
detected with events, copied back, and their slots and memory returned.

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
    """HBM one member of a batched CGLS keeps resident: x, p, s
    (volume-sized) and b, r, q (projection-sized) in elem-byte values; the
    forward projector's quads of the two zero-bordered layouts and the
    backprojector's quads of the zero-bordered projections (two border
    columns a side, and the rows the volume's shadow reaches beyond the
    detector, taken as 10 % + 8), four FP32 coefficients (16 bytes) per
    padded voxel or pixel whatever elem is; plus 64 MiB of slack."""
    nx, ny, nz = geo["n_voxel"]
    nu, nv = geo["n_det"]
    vol = elem * nx * ny * nz
    vol_quads = 2 * 16 * (nx + 4) * (ny + 4) * (nz + 4)
    proj = elem * nu * nv * n_angles
    proj_quads = 16 * n_angles * (nu + 4) * (nv + nv // 10 + 8)
    return 3 * vol + 3 * proj + proj_quads + vol_quads + (64 << 20)


_STORAGE = (torch.float32, torch.bfloat16, torch.float16)


def storage_dtype(req: Request) -> torch.dtype:
    return req.proj.dtype if req.proj.dtype in _STORAGE else torch.float32


def request_bytes(req: Request) -> int:
    return footprint_bytes(req.geo, len(req.angles), storage_dtype(req).itemsize)


def batch_key(req: Request) -> tuple:
    """Requests with equal keys can share one batched CGLS: same geometry,
    angles, storage type and iteration count."""
    geo = tuple(sorted((k, tuple(v) if isinstance(v, (list, tuple)) else v)
                       for k, v in req.geo.items()))
    ang = np.ascontiguousarray(req.angles, dtype=np.float64).tobytes()
    return geo, ang, storage_dtype(req), req.n_iter


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
    return [g[0] for g in admit_groups(queue, n_active, used, max_slots, budget, policy, 1)]


def admit_groups(queue: list[Request], n_active: int, used: int, max_slots: int, budget: int,
                 policy: str = "fifo", max_batch: int = 1) -> list[list[Request]]:
    """As `admit`, in groups: each admitted request (the head of the queue in
    turn) takes along the requests queued behind it with its batch_key, up to
    max_batch per group, while slots (one per request) and HBM remain."""
    if policy == "sjf":
        queue.sort(key=lambda r: (work_estimate(r), r.arrival, r.rid))
    out: list[list[Request]] = []
    n = n_active
    while queue and n < max_slots:
        need = request_bytes(queue[0])
        if used + need > budget and n > 0:
            break
        head = queue.pop(0)
        group = [head]
        used += need
        n += 1
        key = batch_key(head)
        i = 0
        while len(group) < max_batch and i < len(queue) and n < max_slots:
            r = queue[i]
            if batch_key(r) == key and used + request_bytes(r) <= budget:
                group.append(queue.pop(i))
                used += request_bytes(r)
                n += 1
            else:
                i += 1
        out.append(group)
    return out


@dataclass
class _Slot:
    reqs: list
    G: tigre.Geometry
    stream: torch.cuda.Stream
    b: list
    x: list
    state: object
    issued: int
    admitted: float
    done_event: torch.cuda.Event = field(default_factory=lambda: torch.cuda.Event())
    bytes: int = 0

    @property
    def n_iter(self) -> int:
        return self.reqs[0].n_iter


class Server:
    def __init__(self, max_slots: int = 8, hbm_budget: int | None = None, graph: bool = True,
                 iters_per_tick: int = 2, device: int = 0, policy: str = "fifo",
                 max_batch: int = 4):
        """policy: "fifo" admits in arrival order; "sjf" admits the queued
        request with the least estimated work (voxels x angles x iterations)
        first, which shortens the typical latency when big and small
        reconstructions are mixed.  max_batch: the most requests of one
        batch key run as one batched CGLS (1: every request alone)."""
        if policy not in ("fifo", "sjf"):
            raise ValueError("policy must be 'fifo' or 'sjf'")
        self.policy = policy
        self.max_batch = max(1, int(max_batch))
        self.groups: list[list[int]] = []  # request ids of every group admitted, in order
        self.max_slots = max_slots
        self.graph = graph
        self.iters_per_tick = max(1, iters_per_tick)
        self.device = torch.device("cuda", device)
        if hbm_budget is None:
            free, _ = torch.cuda.mem_get_info(self.device)
            hbm_budget = int(0.8 * free)
        self.hbm_budget = hbm_budget

    def _admit(self, group: list[Request], now: float) -> _Slot:
        stream = torch.cuda.Stream(device=self.device)
        head = group[0]
        self.groups.append([r.rid for r in group])
        with torch.cuda.stream(stream):
            G = tigre.Geometry(head.geo, head.angles)
            dt = storage_dtype(head)
            bs = [r.proj.to(self.device, dtype=dt, non_blocking=True) for r in group]
            # zeroed by the library (zero start: r = b, no projection of x0)
            xs = [torch.empty(G.vol_shape, device=self.device, dtype=dt) for _ in group]
            state = tigre.tigre_cgls_batch_begin(G.handle, bs, xs, n_iter_hint=head.n_iter,
                                                 stream=stream, graph=self.graph, x0_zero=True)
        return _Slot(group, G, stream, bs, xs, state, 0, now,
                     bytes=sum(request_bytes(r) for r in group))

    def _finish(self, s: _Slot, now: float) -> list[Result]:
        out = []
        for i, r in enumerate(s.reqs):
            resid = tigre.tigre_cgls_batch_history(s.state, i, r.n_iter)  # syncs the stream
            out.append(Result(r.rid, s.x[i].float().cpu(), resid, r.arrival, s.admitted, now))
        tigre.tigre_cgls_batch_end(s.state)
        s.G.close()
        return out

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
            # work first), same-key requests grouped into one batch.
            n_active = sum(len(s.reqs) for s in active)
            for group in admit_groups(queue, n_active, used, self.max_slots, self.hbm_budget,
                                      self.policy, self.max_batch):
                slot = self._admit(group, time.perf_counter() - t0)
                used += slot.bytes
                active.append(slot)
            # One tick of work for every resident group.
            for s in active:
                if s.issued < s.n_iter:
                    n = min(self.iters_per_tick, s.n_iter - s.issued)
                    with torch.cuda.stream(s.stream):
                        tigre.tigre_cgls_batch_iterate(s.state, n)
                    s.issued += n
                    if s.issued == s.n_iter:
                        s.done_event.record(s.stream)
            # Retire finished groups.
            still = []
            for s in active:
                if s.issued == s.n_iter and s.done_event.query():
                    results.extend(self._finish(s, time.perf_counter() - t0))
                    used -= s.bytes
                else:
                    still.append(s)
            active = still
            if not active and not queue and pending and realtime:
                time.sleep(max(0.0, pending[0].arrival - (time.perf_counter() - t0)))
            elif active and all(s.issued == s.n_iter for s in active):
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
