"""Serving benchmark: a Poisson stream of CBCT reconstruction requests served
by the continuous-batching server versus the one-at-a-time plain path.

    python -m paper_1905_03748_gb300.serving_bench [--n 16] [--rate 20] [--seed 5]

Requests: volumes 128^3-512^3 (256 mm field of view), detectors 256^2-768^2
sized to the shadow, 90-720 angles, projections uploaded as FP32 or BF16,
15 CGLS iterations each, seeded random-ellipsoid phantoms.  Prints one JSON
line: p50 / p99 latency, makespan and throughput for both paths, and the
largest difference between a request's result in the two runs.
"""
from __future__ import annotations

import argparse
import json

import numpy as np
import torch

from . import serving, synth, tigre


def build_requests(n: int, rate: float, seed: int, n_iter: int):
    sizes = [128, 192, 256, 384, 512]
    probs = [0.3, 0.25, 0.2, 0.15, 0.1]

    def make(i, rng):
        nv = int(rng.choice(sizes, p=probs))
        det = int(min(768, max(256, round(1.5 * nv / 64) * 64)))
        na = int(rng.choice([90, 180, 360, 720] if nv <= 256 else [90, 180, 360]))
        geo = synth.cube_geometry(nv, det)
        ang = synth.angles(na)
        vol = synth.voxelize(synth.random_ellipsoids(nv, 256.0 / nv, 12, seed=1000 + i),
                             geo["n_voxel"], geo["d_voxel"])
        with tigre.Geometry(geo, ang) as G:
            b = G.forward(torch.from_numpy(vol).cuda())
        dtype = torch.bfloat16 if rng.random() < 0.5 else torch.float32
        return geo, ang, b.to(dtype).cpu().pin_memory(), n_iter

    return serving.poisson_requests(n, rate, seed, make)


def work(reqs):
    return sum(2.0 * np.prod(r.geo["n_voxel"]) * len(r.angles) * (r.n_iter + 1) for r in reqs)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=24)
    ap.add_argument("--rate", type=float, default=20.0)
    ap.add_argument("--seed", type=int, default=5)
    ap.add_argument("--iters", type=int, default=15)
    ap.add_argument("--slots", type=int, default=6)
    a = ap.parse_args()
    reqs = build_requests(a.n, a.rate, a.seed, a.iters)
    torch.cuda.synchronize()
    # warm both paths on one small request (module load, first allocations)
    serving.run_plain(reqs[:1], realtime=False)
    plain = serving.run_plain(reqs, realtime=True)
    by_id = {r.rid: r for r in plain}
    total = work(reqs)
    sp = serving.latency_stats(plain)
    out = {"requests": a.n, "rate_per_s": a.rate, "cgls_iters": a.iters,
           "sizes": sorted(int(r.geo["n_voxel"][0]) for r in reqs),
           "plain": dict(sp, gvox_ang_s=total / sp["makespan_s"] / 1e9)}
    for policy in ("fifo", "sjf"):
        server = serving.Server(max_slots=a.slots, graph=True, iters_per_tick=2, policy=policy)
        mixed = server.run(reqs, realtime=True)
        sm = serving.latency_stats(mixed)
        out[f"continuous_batching_{policy}"] = dict(
            sm, gvox_ang_s=total / sm["makespan_s"] / 1e9, slots=a.slots,
            p50_speedup=sp["p50_s"] / sm["p50_s"], p99_speedup=sp["p99_s"] / sm["p99_s"],
            throughput_ratio=sm["throughput_req_s"] / sp["throughput_req_s"],
            max_abs_diff_vs_alone=max(float((r.x - by_id[r.rid].x).abs().max()) for r in mixed))
    print(json.dumps(out))


if __name__ == "__main__":
    main()
