"""Out-of-core CGLS on one GPU at full size (Alg. 1 / Alg. 2 splitting recast
as z-slab streaming), end to end through the public API.

Steps, each timed:
1. a seeded random-ellipsoid phantom (50 ellipsoids, seed 4) generated slab
   by slab into a host buffer;
2. b = A x_true with tigre_forward_ooc (host volume streamed in z-slabs);
   b is copied to a host buffer;
3. tigre_cgls with TIGRE_OUT_OF_CORE from x0 = 0, reusing the phantom's host
   buffer for x (the only volume-sized host allocation);
4. the relative error of x against the phantom, regenerated slab by slab.

Before allocating, the host and device needs are checked against what the
machine has (MemAvailable and the cgroup limit; cudaMemGetInfo) and the run
stops with a message when they do not fit with a margin.

    python -m paper_1905_03748_gb300.ooc_cgls_bench --workload ooc_3072 --iters 10
    python -m paper_1905_03748_gb300.ooc_cgls_bench --n 512 --angles 360 --iters 3 --budget-gb 2
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import torch

from . import synth
from . import tigre as T


def host_available_bytes() -> int:
    """Smaller of MemAvailable and the cgroup's remaining limit."""
    avail = None
    with open("/proc/meminfo") as f:
        for line in f:
            if line.startswith("MemAvailable:"):
                avail = int(line.split()[1]) * 1024
    limits = [avail] if avail is not None else []
    for lim, cur in (("/sys/fs/cgroup/memory.max", "/sys/fs/cgroup/memory.current"),
                     ("/sys/fs/cgroup/memory/memory.limit_in_bytes",
                      "/sys/fs/cgroup/memory/memory.usage_in_bytes")):
        try:
            with open(lim) as f:
                v = f.read().strip()
            with open(cur) as f:
                c = int(f.read().strip())
            if v != "max" and int(v) < (1 << 60):
                limits.append(int(v) - c)
        except (OSError, ValueError):
            pass
    return min(limits) if limits else 0


def stage(msg: str) -> None:
    """Progress line on stderr (kept when a long run is cut short)."""
    print(f"[ooc_cgls_bench {time.strftime('%H:%M:%S')}] {msg}", file=sys.stderr, flush=True)


def main(argv=None) -> dict:
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--workload", default=None, help="named workload (e.g. ooc_3072)")
    ap.add_argument("--n", type=int, default=512, help="cube size when no workload is named")
    ap.add_argument("--angles", type=int, default=360)
    ap.add_argument("--iters", type=int, default=10)
    ap.add_argument("--budget-gb", type=float, default=0.0,
                    help="device budget for the CGLS (0 = free memory)")
    ap.add_argument("--seed", type=int, default=4)
    ap.add_argument("--slab-gen", type=int, default=64, help="planes per phantom slab")
    ap.add_argument("--host-margin", type=float, default=0.9,
                    help="fraction of available host memory the run may take")
    ap.add_argument("--no-error", action="store_true", help="skip the error pass")
    ap.add_argument("--brick", type=int, default=0,
                    help="x-y brick edge of the slab projections (0 = default)")
    ap.add_argument("--path", type=int, default=0, help="forward kernel path (0 = automatic)")
    ap.add_argument("--out", default=None, help="write the JSON result here too")
    a = ap.parse_args(argv)

    if a.workload:
        geo, ang = synth.workload(a.workload)
        name = a.workload
    else:
        geo, ang = synth.cube_geometry(a.n, a.n), synth.angles(a.angles)
        name = f"cube_{a.n}_{a.angles}"
    nx, ny, nz = geo["n_voxel"]
    nu, nv = geo["n_det"]
    na = len(ang)
    nvox, m = nx * ny * nz, nu * nv * na
    need_host = 4 * (nvox + m)
    avail = host_available_bytes()
    res = {"workload": name, "n_voxel": [nx, ny, nz], "n_det": [nu, nv], "angles": na,
           "iters": a.iters, "host_bytes_needed": need_host, "host_bytes_available": avail,
           "cores": os.cpu_count()}
    if need_host > a.host_margin * avail:
        res["error"] = "host memory too small for x and b"
        print(json.dumps(res))
        return res
    budget = int(a.budget_gb * (1 << 30))
    dev = torch.device("cuda")
    with T.Geometry(geo, ang) as G:
        T.tigre_geometry_set_brick(G.handle, a.brick)
        T.tigre_geometry_set_forward_path(G.handle, a.path)
        placement, slab = T.tigre_cgls_ooc_plan(G.handle, budget)
        res.update(placement=placement, slab_planes=slab, device_budget_bytes=budget,
                   brick=a.brick, path=a.path)
        free_b, total_b = torch.cuda.mem_get_info()
        res["device_bytes_total"] = int(total_b)

        # 1. phantom, slab by slab, into a pageable host buffer (the library
        # page-locks it for each call).
        t0 = time.perf_counter()
        ells = synth.random_ellipsoids(nx, geo["d_voxel"][0], 50, a.seed)
        x = torch.empty((nz, ny, nx), dtype=torch.float32)
        for z0 in range(0, nz, a.slab_gen):
            z1 = min(nz, z0 + a.slab_gen)
            x[z0:z1].copy_(synth.voxelize_torch(ells, (nx, ny, nz), geo["d_voxel"], (z0, z1), dev))
        torch.cuda.synchronize()
        res["t_phantom_s"] = time.perf_counter() - t0
        stage(f"phantom {res['t_phantom_s']:.1f} s; placement {placement}, slab {slab}")

        # 2. b = A x_true, streamed from host memory (Alg. 1)
        torch.cuda.empty_cache()
        bd = torch.empty((na, nv, nu), dtype=torch.float32, device=dev)
        torch.cuda.synchronize()
        T.tigre_profile_enable(True)
        t0 = time.perf_counter()
        T.tigre_forward_ooc(G.handle, x, bd, 0, na)
        torch.cuda.synchronize()
        res["t_forward_ooc_s"] = time.perf_counter() - t0
        res["forward_ooc_kernel_s"] = T.tigre_profile_read(T.PROF_FORWARD)[1] / 1e3
        res["forward_ooc_gvox_ang_per_s"] = nvox * na / res["t_forward_ooc_s"] / 1e9
        stage(f"b = A x_true out of core: {res['t_forward_ooc_s']:.1f} s")
        b = torch.empty((na, nv, nu), dtype=torch.float32)
        b.copy_(bd)
        del bd
        torch.cuda.empty_cache()

        # 3. CGLS from x0 = 0 in the phantom's buffer
        x.zero_()
        T.tigre_profile_enable(True)  # resets the totals
        t0 = time.perf_counter()
        hist = T.tigre_cgls(G.handle, b, x, a.iters, out_of_core=True,
                            device_budget_bytes=budget)
        res["t_cgls_s"] = time.perf_counter() - t0
        # device time of the projection and backprojection kernels inside it:
        # the rest is slab preparation, vector updates and host transfers not
        # hidden behind compute
        res["cgls_forward_kernel_s"] = T.tigre_profile_read(T.PROF_FORWARD)[1] / 1e3
        res["cgls_backproject_kernel_s"] = T.tigre_profile_read(T.PROF_BACKPROJECT)[1] / 1e3
        T.tigre_profile_enable(False)
        res["residual_history"] = [float(v) for v in hist]
        stage(f"cgls {a.iters} iterations: {res['t_cgls_s']:.1f} s")

        # 4. relative error against the phantom
        if not a.no_error:
            t0 = time.perf_counter()
            num = den = 0.0
            finite = True
            for z0 in range(0, nz, a.slab_gen):
                z1 = min(nz, z0 + a.slab_gen)
                xt = synth.voxelize_torch(ells, (nx, ny, nz), geo["d_voxel"], (z0, z1), dev)
                xs = x[z0:z1].to(dev)
                finite = finite and bool(torch.isfinite(xs).all())
                num += float(torch.linalg.vector_norm((xs - xt).double()) ** 2)
                den += float(torch.linalg.vector_norm(xt.double()) ** 2)
            res["rel_error_vs_phantom"] = (num / den) ** 0.5 if den > 0 else None
            res["x_finite"] = finite
            res["t_error_s"] = time.perf_counter() - t0
    print(json.dumps(res))
    if a.out:
        with open(a.out, "w") as f:
            json.dump(res, f, indent=1)
    return res


if __name__ == "__main__":
    main()
