#!/usr/bin/env python
"""Benchmark of the iterative cone-beam CT hot path.

Workload (default): 512^3 float32 volume of 0.5 mm voxels holding 50 seeded
random ellipsoids, 512^2 detector, 360 angles over 360 degrees, DSO 1000 mm,
DSD 1536 mm; b = A x_true.  One step = one CGLS iteration: a forward
projection A p, a matched backprojection A^T r and the FP64 inner products
and vector updates, all resident on the GPU.

Metric: Gvoxel*angles/s = 2 * 512^3 * 360 per step / step time (each
operator visits every voxel-angle pair once), plus CGLS s/iter and the
per-operator rates.  Multi-GPU (torchrun): every rank reconstructs its own
problem (independent reconstructions, no data-path collective); the value is
the sum of the work over the max step time across ranks.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Ax/Aᵀy Gvoxel·angles/s and CGLS s/iter at 512³×360"
UNIT = "Gvoxel*angles/s"
FLOPS_PER_SAMPLE = 22  # trilinear interpolation: 7 lerps x 3 flops + 1 accumulation
L1_BYTES_PER_SAMPLE = 32  # the eight FP32 taps a trilinear sample gathers
L1_BYTES_PER_VOXEL_ANGLE = 16  # the four FP32 taps a backprojected voxel-angle gathers
KERNEL_SOURCES = ["paper_1905_03748_gb300/csrc/forward.cu", "paper_1905_03748_gb300/csrc/ray.cuh",
                  "paper_1905_03748_gb300/csrc/quad.cuh"]
BP_SOURCES = ["paper_1905_03748_gb300/csrc/backward.cu", "paper_1905_03748_gb300/csrc/ray.cuh",
              "paper_1905_03748_gb300/csrc/quad.cuh"]
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "fwd_kernel_traffic.json")
BP_SOL_FILE = os.path.join(ROOT, "profiles", "bp_kernel_sol.json")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--e2e-iters", type=int, default=20, help="CGLS iterations per e2e call")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-angles", type=int, default=48,
                    help="angles of the workload in the bounded CPU-oracle sample")
    ap.add_argument("--workload", default="cgls_512", choices=["cgls_512", "small_64"],
                    help="cgls_512: the benchmark line (default); small_64: the 64^3 x 100 "
                         "SIRT workload, timed with the oracle beside it")
    return ap.parse_args()


def workload():
    from paper_1905_03748_gb300 import synth
    geo, ang = synth.workload("cgls_512")
    return geo, ang


def config_dict(geo, ang):
    nx, ny, nz = geo["n_voxel"]
    nu, nv = geo["n_det"]
    return {"workload": f"CGLS at {nx}x{ny}x{nz} float32 vol (0.5 mm), {nu}x{nv} det "
                        f"({geo['d_det'][0]:.4f} mm), {len(ang)} angles, DSO 1000 / DSD 1536 mm",
            "step": "one CGLS iteration (Ax + matched A^T y + FP64 dots/updates)",
            "l2": "inputs larger than L2 (vol 512 MiB, proj 360 MiB > 126 MB L2): no flush",
            "phantom": "50 seeded random ellipsoids (seed 2), b = A x_true"}


def source_hash(sources=KERNEL_SOURCES) -> str:
    h = hashlib.sha256()
    for p in sources:
        with open(os.path.join(ROOT, p), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                                         text=True)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        self.out = ""
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in (self.out or "").splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_init(backend):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws <= 1:
        return 0, 1, None
    import torch.distributed as dist
    dist.init_process_group(backend=backend)
    return dist.get_rank(), ws, dist


def max_over_ranks(x: float, dist, device=None) -> float:
    """Largest value of x over all ranks (the job's step time); identity
    without a process group.  No data-path collective: timings only."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(work_per_rank: float, world: int, seconds: float) -> float:
    """Whole-job throughput for independent per-rank problems (weak
    scaling): all ranks' work over the slowest rank's time, in G/s."""
    return world * work_per_rank / seconds / 1e9


def cpu_baseline(geo, ang, x_true, n_angles):
    """The FP64 oracle, as it stands, on a bounded sample of the workload:
    one forward projection and one matched backprojection over the first
    n_angles angles (the per-step operators of CGLS)."""
    import oracle
    oracle.build()
    sub = ang[:n_angles]
    xv = np.asarray(x_true, dtype=np.float64)
    t0 = time.perf_counter()
    p = oracle.forward(geo, sub, xv)
    oracle.backward(geo, sub, p, oracle.BP_MATCHED)
    dt = time.perf_counter() - t0
    nvox = int(np.prod(geo["n_voxel"]))
    return {"value": 2.0 * nvox * n_angles / dt / 1e9, "unit": UNIT, "cores": os.cpu_count(),
            "kind": "oracle",
            "sample": f"FP64 oracle Ax + matched A^T y over {n_angles} of {len(ang)} angles of "
                      f"the 512^3 workload ({dt:.1f} s)"}


def run_reference(args):
    """Reference arm: the FP64 CPU oracle timed on the host cores."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_1905_03748_gb300 import synth
    geo, ang = workload()
    x_true = synth.phantom("ellipsoids50", 512, 0.5, seed=2, dtype=np.float64)
    import oracle
    oracle.build()
    n_sub = 2
    nvox = int(np.prod(geo["n_voxel"]))

    def step(i):
        sub = ang[(2 * i) % len(ang):(2 * i) % len(ang) + n_sub]
        p = oracle.forward(geo, sub, x_true)
        oracle.backward(geo, sub, p, oracle.BP_MATCHED)

    for i in range(args.warmup):
        step(i)
    t0 = time.perf_counter()
    for i in range(args.steps):
        step(args.warmup + i)
    dt = (time.perf_counter() - t0) / args.steps
    value = 2.0 * nvox * n_sub / dt / 1e9
    sample = (f"each step: FP64 oracle Ax + matched A^T y over {n_sub} of {len(ang)} angles "
              f"of the 512^3 workload")
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
           "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": dt * 1e3, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": config_dict(geo, ang),
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": os.cpu_count(),
                            "kind": "oracle", "sample": sample},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def run_ours(args):
    import torch
    from paper_1905_03748_gb300 import synth, tigre

    rank, world, dist = dist_init("nccl")
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    geo, ang = workload()
    nx, ny, nz = geo["n_voxel"]
    nvox = nx * ny * nz
    x_np = synth.phantom("ellipsoids50", 512, 0.5, seed=2 + rank)
    G = tigre.Geometry(geo, ang)
    x_true = torch.from_numpy(x_np).to(dev)
    b = G.forward(x_true)
    torch.cuda.synchronize()
    x = torch.zeros(G.vol_shape, device=dev)
    state = tigre.tigre_cgls_begin(G.handle, b, x, n_iter_hint=args.warmup + args.steps)
    tigre.tigre_cgls_iterate(state, args.warmup)
    torch.cuda.synchronize()

    stream = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(torch.cuda.current_device()) as clk:
        tigre.tigre_profile_enable(True)
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        e0.record(stream)
        tigre.tigre_cgls_iterate(state, args.steps)
        e1.record(stream)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
    launches = tigre.tigre_launch_count()
    fwd_n, fwd_ms = tigre.tigre_profile_read(tigre.PROF_FORWARD)
    bp_n, bp_ms = tigre.tigre_profile_read(tigre.PROF_BACKPROJECT)
    tigre.tigre_profile_enable(False)
    ms = max_over_ranks(e0.elapsed_time(e1) / args.steps, dist, dev)
    hist = tigre.tigre_cgls_history(state, args.warmup + args.steps)
    tigre.tigre_cgls_end(state)

    vox_ang = float(nvox) * len(ang)
    value = job_rate(2.0 * vox_ang, world, ms / 1e3)
    samples = tigre.tigre_forward_samples(G.handle, 0, len(ang))
    fwd_avg = fwd_ms / max(fwd_n, 1)
    bp_avg = bp_ms / max(bp_n, 1)
    peaks = measured_peaks()
    sm_max_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    fp32_peak = n_sm * 128 * 2 * sm_max_mhz * 1e6 / 1e12  # TFLOP/s, FMA = 2 flops
    alu_achieved = samples * FLOPS_PER_SAMPLE / (fwd_avg / 1e3) / 1e12
    l1_peak = n_sm * 128 * sm_max_mhz * 1e6 / 1e12  # TB/s: 128 B per SM per clock
    l1_achieved = samples * L1_BYTES_PER_SAMPLE / (fwd_avg / 1e3) / 1e12
    traffic = None
    sol = None
    try:
        with open(TRAFFIC_FILE) as f:
            tr = json.load(f)
        if tr.get("source_hash") == source_hash():
            traffic = tr.get("dram_bytes_per_launch")
            sol = tr.get("ncu_sol")
    except Exception:
        pass
    bp_sol = None
    try:
        with open(BP_SOL_FILE) as f:
            tr = json.load(f)
        if tr.get("source_hash") == source_hash(BP_SOURCES):
            bp_sol = tr.get("ncu_sol")
    except Exception:
        pass
    bp_l1 = vox_ang * L1_BYTES_PER_VOXEL_ANGLE / (bp_avg / 1e3) / 1e12

    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": config_dict(geo, ang),
           "cgls_s_per_iter": ms / 1e3,
           "ax_kernel_gvox_ang_s": vox_ang / (fwd_avg / 1e3) / 1e9,
           "atb_kernel_gvox_ang_s": vox_ang / (bp_avg / 1e3) / 1e9,
           "ax_gsamples_s": samples / (fwd_avg / 1e3) / 1e9,
           "samples_per_ax": samples,
           "kernel_ms": {"forward": fwd_avg, "backproject_matched": bp_avg},
           "resid_last": float(hist[-1]) if len(hist) else None,
           "roofline": {"kernel": "fwd_quad_kernel", "bound": "l1", "achieved": l1_achieved,
                        "peak": l1_peak, "unit": "TB/s", "frac": l1_achieved / l1_peak,
                        "traffic": traffic,
                        "per_unit": f"{L1_BYTES_PER_SAMPLE} B gathered per quadrature sample "
                                    f"(eight FP32 taps) x {samples} samples per launch",
                        "peak_source": f"{n_sm} SMs (device query) x 128 B per clock (L1 data "
                                       f"path) x max SM clock {sm_max_mhz:.0f} MHz (derived; "
                                       "no measured L1 peak exists)",
                        "binding_unit": "L1/TEX data path (gathers), not DRAM, not the FP32 pipe",
                        "ncu_sol": sol,
                        "alu": {"achieved_tflops": alu_achieved, "peak_tflops": fp32_peak,
                                "frac": alu_achieved / fp32_peak,
                                "per_unit": f"{FLOPS_PER_SAMPLE} FP32 flops per sample",
                                "peak_source": f"{n_sm} SMs x 128 FP32 lanes x 2 x "
                                               f"{sm_max_mhz:.0f} MHz (derived)"}},
           "roofline_backprojector": {"kernel": "bp_voxel_kernel (matched)", "bound": "l1",
                                      "achieved": bp_l1, "peak": l1_peak, "unit": "TB/s",
                                      "frac": bp_l1 / l1_peak,
                                      "per_unit": f"{L1_BYTES_PER_VOXEL_ANGLE} B gathered per "
                                                  "voxel-angle (four FP32 taps)",
                                      "ncu_sol": bp_sol},
           "gpu_launches": launches, "clocks": clk.summary(),
           "paper_context": "CGLS 512^3, 15 it in 61 s (4.1 s/iter incl. host copies), "
                            "1x GTX 1080 Ti (Sec. 4); detector/angles not stated"}

    if not args.no_e2e:
        n_e2e = args.e2e_iters
        bh = b.cpu().pin_memory()
        xh = torch.zeros(G.vol_shape).pin_memory()
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        tigre.tigre_cgls(G.handle, bh, xh, n_e2e, host=True, x0_zero=True)
        dt = max_over_ranks(time.perf_counter() - t0, dist, dev)
        out["e2e"] = {"value": job_rate(2.0 * vox_ang * n_e2e, world, dt), "unit": UNIT,
                      "h2d_bytes_per_step": bh.numel() * 4,
                      "d2h_bytes_per_step": xh.numel() * 4,
                      "step": f"tigre_cgls call on pinned host buffers from x0 = 0: copy b in, "
                              f"{n_e2e} CGLS iterations (+ initial r = b, A^T r), copy x out",
                      "s_per_call": dt}
    if rank == 0 and world == 1 and not args.no_cpu:
        out["cpu_baseline"] = cpu_baseline(geo, ang, x_np, args.cpu_angles)
    G.close()
    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist:
        dist.destroy_process_group()


def run_small(args):
    """The 64^3 workload: 64^3 volume of 1 mm voxels (nested 10-ellipsoid
    head stand-in), 128^2 detector of 0.8 mm, 100 angles.  One step = one
    forward projection, one matched backprojection and a 10-iteration SIRT
    solve from x0 = 0, device-timed with CUDA events (launch bound at this
    size, so wall time per step and the launch count are what is reported).
    The oracle does the same work on the host cores beside it."""
    import torch
    from paper_1905_03748_gb300 import synth, tigre

    torch.cuda.set_device(0)
    geo, ang = synth.workload("small_64")
    x_np = synth.phantom("head10", 64, 1.0)
    G = tigre.Geometry(geo, ang)
    xt = torch.from_numpy(x_np).cuda()
    b = G.forward(xt)
    x = torch.zeros(G.vol_shape, device="cuda")
    stream = torch.cuda.current_stream()
    n_sirt = 10

    def step():
        p = G.forward(xt)
        G.backward(p, weight="matched")
        tigre.tigre_sirt(G.handle, b, x, n_sirt, stream=stream.cuda_stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    l0 = tigre.tigre_launch_count()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(torch.cuda.current_device()) as clk:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e0.record(stream)
        for _ in range(args.steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
        wall = (time.perf_counter() - t0) / args.steps
    ms = e0.elapsed_time(e1) / args.steps
    launches = (tigre.tigre_launch_count() - l0) // args.steps
    vox_ang = float(np.prod(geo["n_voxel"])) * len(ang)
    work = vox_ang * (2 + 2 * n_sirt) + vox_ang  # FP + BP + (FP + BP) per SIRT it + W = A 1
    out = {"metric": "64^3 x 100: FP + matched BP + 10 SIRT iterations, s per step",
           "value": ms / 1e3, "unit": "s/step", "n_gpus": 1, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": "64^3 vol (1 mm, nested 10-ellipsoid stand-in for the modified "
                                  "Shepp-Logan head), 128^2 det (0.8 mm), 100 angles, DSO 1000 / "
                                  "DSD 1536 mm",
                      "step": "A x, matched A^T y, then tigre_sirt 10 iterations from x0 = 0",
                      "l2": "working set fits L2 (launch-bound size)"},
           "sirt_ms_per_iter_incl_setup": None, "host_wall_ms_per_step": wall * 1e3,
           "gvox_ang_s": work / (ms / 1e3) / 1e9, "gpu_launches_per_step": launches,
           "clocks": clk.summary()}
    # SIRT alone, for the per-iteration figure
    torch.cuda.synchronize()
    e0.record(stream)
    tigre.tigre_sirt(G.handle, b, x, n_sirt, stream=stream.cuda_stream)
    e1.record(stream)
    torch.cuda.synchronize()
    out["sirt_ms_per_iter_incl_setup"] = e0.elapsed_time(e1) / n_sirt
    if not args.no_cpu:
        import oracle
        oracle.build()
        xv = x_np.astype(np.float64)
        t0 = time.perf_counter()
        p = oracle.forward(geo, ang, xv)
        oracle.backward(geo, ang, p, oracle.BP_MATCHED)
        oracle.sirt(geo, ang, b.cpu().numpy(), n_sirt)
        dt = time.perf_counter() - t0
        out["cpu_baseline"] = {"value": dt, "unit": "s/step", "cores": os.cpu_count(),
                               "kind": "oracle",
                               "sample": "the whole step (FP + matched BP + 10 SIRT iterations) "
                                         "by the FP64 oracle"}
    G.close()
    print(json.dumps(out), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "small_64":
        run_small(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
