"""Mixed-precision study: volume / projection storage in FP32, BF16 and FP16
(FP32 accumulation along every ray and voxel sum, FP64 solver scalars).

    python -m paper_1905_03748_gb300.precision_bench [--n 1024] [--angles 720] [--iters 2]
    python -m paper_1905_03748_gb300.precision_bench --solver cgls --n 512 --angles 360 --iters 10

Workload: N^3 volume (256 mm field of view), N^2 detector, A angles, seeded
piecewise-constant phantom (random ellipsoids, seed 3), projections with
Gaussian noise of 1 % of their maximum on every ray that crosses the object
(rays that only graze the support would have their noise multiplied by the
huge SART row weight 1/(A 1)).  For each storage type it reports:
  * forward / backprojection relative difference from the FP32-storage
    result (the error the storage type itself adds);
  * OS-SART (subsets of 20 angles) + TV (20 gradient steps, alpha 0.002)
    reconstruction error against the phantom, and against the FP32 solve,
    plus seconds per iteration;
  * or, with --solver cgls, the same for CGLS with every vector stored in
    the type (FP64 inner products and step lengths); FP16 runs on b scaled
    by 1e-3 to stay inside its range (CGLS is linear in b; x is scaled back).
(The errors against the FP64 oracle are measured by the GPU test suite on
sampled rays and voxels of this workload.)
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np
import torch

from . import synth, tigre

DTYPES = {"f32": torch.float32, "bf16": torch.bfloat16, "f16": torch.float16}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=1024)
    ap.add_argument("--angles", type=int, default=720)
    ap.add_argument("--iters", type=int, default=2)
    ap.add_argument("--solver", choices=["os_sart_tv", "cgls"], default="os_sart_tv")
    a = ap.parse_args()
    geo = synth.cube_geometry(a.n, a.n)
    ang = synth.angles(a.angles)
    d = 256.0 / a.n
    x_true = synth.voxelize(synth.random_ellipsoids(a.n, d, 50, seed=3), geo["n_voxel"],
                            geo["d_voxel"])
    out = {"n": a.n, "angles": a.angles, "iters": a.iters, "solver": a.solver,
           "noise": "1% of max b, seeded, on rays crossing the object",
           "storage": {}}
    with tigre.Geometry(geo, ang) as G:
        xt = torch.from_numpy(x_true).cuda()
        b = G.forward(xt)
        b_np = synth.add_noise(b.cpu().numpy(), 0.01, seed=4, object_only=True)
        b_noisy = torch.from_numpy(b_np).cuda()
        p32 = b
        bp32 = G.backward(b_noisy, weight="matched")
        x32 = None
        for name, dt in DTYPES.items():
            rec = {}
            p = G.forward(xt.to(dt), dtype=torch.float32)
            rec["forward_diff_vs_fp32"] = float(torch.linalg.vector_norm(p - p32) /
                                                torch.linalg.vector_norm(p32))
            bp = G.backward(b_noisy.to(dt), weight="matched", dtype=torch.float32)
            rec["backproject_diff_vs_fp32"] = float(torch.linalg.vector_norm(bp - bp32) /
                                                    torch.linalg.vector_norm(bp32))
            del p, bp
            x = torch.zeros(G.vol_shape, device="cuda", dtype=dt)
            scale = 1e-3 if (a.solver == "cgls" and dt == torch.float16) else 1.0
            bb = (b_noisy * scale).to(dt)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            if a.solver == "cgls":
                h = tigre.tigre_cgls(G.handle, bb, x, a.iters)
            else:
                h = tigre.tigre_sart(G.handle, bb, x, a.iters, subset_size=20, tv_steps=20,
                                     tv_alpha=0.002, tv_eps=1e-8)
            torch.cuda.synchronize()
            rec[f"{a.solver}_s_per_iter"] = (time.perf_counter() - t0) / a.iters
            rec["b_scale"] = scale
            xf = x.float() / scale
            h = [v / scale for v in h]
            rec["recon_err_vs_phantom"] = float(torch.linalg.vector_norm(xf - xt) /
                                                torch.linalg.vector_norm(xt))
            if name == "f32":
                x32 = xf.clone()
            else:
                rec["recon_diff_vs_fp32"] = float(torch.linalg.vector_norm(xf - x32) /
                                                  torch.linalg.vector_norm(x32))
            rec["resid_history"] = [float(v) for v in h]
            rec["bytes_volume"] = x.numel() * x.element_size()
            out["storage"][name] = rec
            del x, bb, xf
            torch.cuda.empty_cache()
    print(json.dumps(out))


if __name__ == "__main__":
    main()
