"""Operator microbenchmark: time one operator of the library on an N^3 volume
with an N^2 detector (cube workload geometry) and a chosen number of angles.

    python -m paper_1905_03748_gb300.opbench --op forward --n 512 --angles 360
    python -m paper_1905_03748_gb300.opbench --op backward --weight matched --n 512 --angles 16 --repeat 1

Prints one JSON line: device ms per call (CUDA events on the launching
stream, after one warm-up call), Gvoxel*angles/s, and the projection or
backprojection kernels' own device time per call (the library's event
timer; for the out-of-core operators it excludes the host copies and the
slab relayouts).  Also the small-case target of the committed ncu profiles.
"""
from __future__ import annotations

import argparse
import json
import os
import tempfile

import numpy as np
import torch

from . import synth, tigre


def cached_phantom(n: int) -> np.ndarray:
    """The 50-ellipsoid phantom, kept in the temp directory between runs (its
    numpy voxelisation takes seconds at 512^3)."""
    path = os.path.join(tempfile.gettempdir(), f"tigre103_ellipsoids50_{n}.npy")
    if os.path.exists(path):
        return np.load(path)
    vol = synth.phantom("ellipsoids50", n, 256.0 / n)
    np.save(path + ".tmp.npy", vol)
    os.replace(path + ".tmp.npy", path)
    return vol


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--op", choices=["forward", "backward", "adjoint", "tv", "forward_ooc",
                                     "backward_ooc", "fdk", "rof"], default="forward")
    ap.add_argument("--slab", type=int, default=0, help="out-of-core slab planes (0 = auto)")
    ap.add_argument("--weight", choices=["matched", "fdk"], default="matched")
    ap.add_argument("--n", type=int, default=512)
    ap.add_argument("--angles", type=int, default=360)
    ap.add_argument("--dtype", choices=["f32", "bf16", "f16"], default="f32")
    ap.add_argument("--repeat", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=1)
    ap.add_argument("--path", choices=["auto", "l1", "tma", "quad", "pair", "ag2", "ag4"],
                    default="auto",
                    help="forward-projector kernel")
    ap.add_argument("--projector", choices=["interpolated", "siddon"], default="interpolated")
    ap.add_argument("--brick", type=int, default=0,
                    help="x-y brick edge of slab projections (0 = library default)")
    a = ap.parse_args()
    dt = {"f32": torch.float32, "bf16": torch.bfloat16, "f16": torch.float16}[a.dtype]
    geo = synth.cube_geometry(a.n, a.n)
    ang = synth.angles(a.angles)
    G = tigre.Geometry(geo, ang)
    tigre.tigre_geometry_set_forward_path(G.handle, {"auto": 0, "l1": 1, "tma": 2, "quad": 3,
                                                     "pair": 4, "ag2": 5, "ag4": 6}[a.path])
    tigre.tigre_geometry_set_projector(G.handle, a.projector)
    tigre.tigre_geometry_set_brick(G.handle, a.brick)
    vol = torch.from_numpy(cached_phantom(a.n)).cuda().to(dt)
    proj = torch.empty(G.proj_shape, device="cuda", dtype=dt)
    out = torch.empty(G.vol_shape, device="cuda", dtype=dt)
    if a.op in ("backward", "adjoint", "backward_ooc"):
        G.forward(vol, out=proj)
    if a.op in ("forward_ooc", "backward_ooc"):
        vol_host = vol.float().cpu().pin_memory()
        out_host = torch.empty(G.vol_shape, dtype=torch.float32).pin_memory()
    if a.op == "forward":
        fn = lambda: G.forward(vol, out=proj)  # noqa: E731
    elif a.op == "forward_ooc":
        fn = lambda: tigre.tigre_forward_ooc(G.handle, vol_host, proj, 0, a.angles,  # noqa
                                             slab_planes=a.slab)
    elif a.op == "backward_ooc":
        fn = lambda: tigre.tigre_backward_ooc(G.handle, proj, out_host, 0, a.angles,  # noqa
                                              weight=a.weight, slab_planes=a.slab)
    elif a.op == "backward":
        fn = lambda: G.backward(proj, out=out, weight=a.weight)  # noqa: E731
    elif a.op == "adjoint":
        fn = lambda: G.backward(proj, out=out, weight="adjoint")  # noqa: E731
    elif a.op == "fdk":
        G.forward(vol, out=proj)
        fn = lambda: G.fdk(proj, out=out)  # noqa: E731
    elif a.op == "rof":
        volf = vol.float()
        out = torch.empty_like(volf)
        fn = lambda: tigre.tigre_rof_denoise(volf, 20.0, 10, out=out)  # noqa: E731
    else:
        fn = lambda: tigre.tigre_tv_step(vol, 1, 0.002, 1e-8)  # noqa: E731
    for _ in range(a.warmup):
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    tigre.tigre_profile_enable(True)
    e0.record()
    for _ in range(a.repeat):
        fn()
    e1.record()
    torch.cuda.synchronize()
    kind = {"forward": tigre.PROF_FORWARD, "forward_ooc": tigre.PROF_FORWARD,
            "backward": tigre.PROF_BACKPROJECT, "backward_ooc": tigre.PROF_BACKPROJECT,
            "fdk": tigre.PROF_BACKPROJECT, "adjoint": tigre.PROF_ADJOINT}.get(a.op, tigre.PROF_TV)
    kernel_ms = tigre.tigre_profile_read(kind)[1] / max(a.repeat, 1)
    tigre.tigre_profile_enable(False)
    ms = e0.elapsed_time(e1) / max(a.repeat, 1)
    va = float(a.n) ** 3 * a.angles
    print(json.dumps({"op": a.op, "weight": a.weight, "n": a.n, "angles": a.angles,
                      "dtype": a.dtype, "path": a.path, "projector": a.projector, "brick": a.brick, "ms": ms,
                      "kernel_ms": kernel_ms, "gvox_ang_s": va / ms / 1e6,
                      "error_flags": tigre.tigre_geometry_error_flags(G.handle),
                      "checksum": float(proj.float().sum() if a.op in ("forward", "forward_ooc") else
                                        out.float().sum())}))
    G.close()


if __name__ == "__main__":
    main()
