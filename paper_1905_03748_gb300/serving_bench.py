"""Serving benchmark: a Poisson stream of CBCT reconstruction requests served
by the continuous-batching server versus the one-at-a-time plain path.

    python -m paper_1905_03748_gb300.serving_bench [--n 16] [--rate 20] [--seed 5]

Requests follow six scan protocols (volume, detector, angles, storage type),
drawn with fixed probabilities: 128^3 / 256^2 / 90 angles / BF16,
128^3 / 256^2 / 360 / F32, 192^3 / 320^2 / 180 / F32, 256^3 / 384^2 / 360 /
BF16, 384^3 / 576^2 / 360 / F32 and 512^3 / 768^2 / 720 / BF16 (256 mm field
of view, detectors sized to the shadow), 15 CGLS iterations each, seeded
random-ellipsoid phantoms (12 ellipsoids, a different phantom per request).
Paths: one request at a time (tigre_cgls); the server without batching
(max_batch 1: every request its own CGLS, overlapping on streams); the server
grouping same-protocol requests into batched CGLS (max_batch 4), with FIFO
and least-work-first admission.  Prints one JSON line: p50 / p99 latency,
makespan and throughput per path, the groups formed, and the largest
difference between a request's result in the server and alone.
"""
from __future__ import annotations

import argparse
import json

import numpy as np
import torch

from . import serving, synth, tigre


# (volume edge, detector edge, angles, storage type, probability)
PROTOCOLS = [(128, 256, 90, torch.bfloat16, 0.25), (128, 256, 360, torch.float32, 0.15),
             (192, 320, 180, torch.float32, 0.20), (256, 384, 360, torch.bfloat16, 0.20),
             (384, 576, 360, torch.float32, 0.10), (512, 768, 720, torch.bfloat16, 0.10)]


def build_requests(n: int, rate: float, seed: int, n_iter: int):
    probs = [p[4] for p in PROTOCOLS]

    def make(i, rng):
        nv, det, na, dtype, _ = PROTOCOLS[int(rng.choice(len(PROTOCOLS), p=probs))]
        geo = synth.cube_geometry(nv, det)
        ang = synth.angles(na)
        vol = synth.voxelize(synth.random_ellipsoids(nv, 256.0 / nv, 12, seed=1000 + i),
                             geo["n_voxel"], geo["d_voxel"])
        with tigre.Geometry(geo, ang) as G:
            b = G.forward(torch.from_numpy(vol).cuda())
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
    ap.add_argument("--slots", type=int, default=8)
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
           "protocols": [f"{p[0]}^3/{p[1]}^2/{p[2]}/{str(p[3]).split('.')[-1]}/{p[4]}"
                         for p in PROTOCOLS],
           "sizes": sorted(int(r.geo["n_voxel"][0]) for r in reqs),
           "plain": dict(sp, gvox_ang_s=total / sp["makespan_s"] / 1e9)}
    for name, policy, max_batch in (("streams_fifo", "fifo", 1), ("batched_fifo", "fifo", 4),
                                     ("batched_sjf", "sjf", 4)):
        server = serving.Server(max_slots=a.slots, graph=True, iters_per_tick=2, policy=policy,
                                max_batch=max_batch)
        mixed = server.run(reqs, realtime=True)
        sm = serving.latency_stats(mixed)
        out[name] = dict(
            sm, gvox_ang_s=total / sm["makespan_s"] / 1e9, slots=a.slots, max_batch=max_batch,
            groups=[len(g) for g in server.groups],
            p50_speedup=sp["p50_s"] / sm["p50_s"], p99_speedup=sp["p99_s"] / sm["p99_s"],
            throughput_ratio=sm["throughput_req_s"] / sp["throughput_req_s"],
            max_abs_diff_vs_alone=max(float((r.x - by_id[r.rid].x).abs().max()) for r in mixed))
    print(json.dumps(out))


if __name__ == "__main__":
    main()
