"""The workspace allocator hook: every device workspace the library makes goes
through the installed pair (here PyTorch's caching allocator), each is freed,
and results are the same as with the CUDA default (bitwise, except the exact
adjoint, whose FP32 atomic sums vary in order from run to run)."""
import gc

import numpy as np
import pytest
import torch

from paper_1905_03748_gb300 import synth

pytestmark = pytest.mark.gpu


def run_all(tigre):
    geo = synth.geometry((37, 29, 21), (1.0, 0.9, 1.1), (53, 27), (1.05, 0.95), dso=300.0,
                         dsd=450.0, off_origin=(0.5, -0.3, 0.2))
    ang = np.sort(np.random.default_rng(4).uniform(0, 2 * np.pi, 23))
    vol = torch.from_numpy(synth.random_volume((21, 29, 37), seed=5)).cuda()
    out = {}
    with tigre.Geometry(geo, ang) as G:
        p = G.forward(vol)
        out["forward"] = p
        out["matched"] = G.backward(p)
        out["adjoint"] = G.backward(p, weight="adjoint")
        out["fdk"] = G.fdk(p)
        x = torch.zeros(G.vol_shape, device="cuda")
        out["cgls_hist"] = torch.tensor(tigre.tigre_cgls(G.handle, p, x, 3))
        out["cgls"] = x
        t = vol.clone()
        tigre.tigre_tv_step(t, 2, 0.01, 1e-8)
        out["tv"] = t
        out["rof"] = tigre.tigre_rof_denoise(vol, 2.0, 5)
    torch.cuda.synchronize()
    return out


def test_workspaces_go_through_the_installed_allocator(tigre):
    gc.collect()  # handles left to the garbage collector by earlier tests
    ref = run_all(tigre)
    counts = {"alloc": 0, "free": 0}

    def alloc(nbytes, stream):
        counts["alloc"] += 1
        return torch.cuda.caching_allocator_alloc(nbytes, device=torch.cuda.current_device(),
                                                  stream=stream)

    def free(ptr, stream):
        counts["free"] += 1
        torch.cuda.caching_allocator_delete(ptr)

    tigre.tigre_set_allocator(alloc, free)
    try:
        got = run_all(tigre)
    finally:
        torch.cuda.synchronize()
        tigre.tigre_set_allocator(None, None)
    assert counts["alloc"] > 10 and counts["alloc"] == counts["free"]
    for k in ref:
        if k == "adjoint":  # FP32 atomics: the summation order differs run to run
            assert float(torch.linalg.vector_norm(ref[k] - got[k]) /
                         torch.linalg.vector_norm(ref[k])) < 1e-6
        else:
            assert torch.equal(ref[k], got[k]), k


def test_allocator_cannot_change_while_a_handle_is_alive(tigre):
    gc.collect()
    geo = synth.geometry(8, 1.0, 12, 1.0, dso=60.0, dsd=90.0)
    with tigre.Geometry(geo, synth.angles(4)):
        with pytest.raises(tigre.TigreError):
            tigre.use_torch_allocator(True)
    tigre.use_torch_allocator(True)
    tigre.use_torch_allocator(False)


@pytest.mark.parametrize("fail_at", [1, 3, 6])
def test_injected_allocation_failure_is_reported_and_leaks_nothing(tigre, fail_at):
    """Host-side fault injection: the allocator refuses its fail_at-th request.
    The call returns TIGRE_ERR_OOM, every buffer handed out is given back, and
    the next call (default allocator) works."""
    gc.collect()
    live = {}
    n = {"calls": 0}

    def alloc(nbytes, stream):
        n["calls"] += 1
        if n["calls"] == fail_at:
            return 0
        p = torch.cuda.caching_allocator_alloc(nbytes, device=torch.cuda.current_device(),
                                               stream=stream)
        live[p] = nbytes
        return p

    def free(ptr, stream):
        live.pop(ptr)
        torch.cuda.caching_allocator_delete(ptr)

    geo = synth.geometry((21, 19, 17), 1.0, (31, 23), 1.0, dso=200.0, dsd=300.0)
    ang = synth.angles(12)
    vol = torch.from_numpy(synth.random_volume((17, 19, 21), seed=25)).cuda()
    tigre.tigre_set_allocator(alloc, free)
    try:
        with pytest.raises(tigre.TigreError) as e:
            with tigre.Geometry(geo, ang) as G:
                b = G.forward(vol)
                x = torch.zeros(G.vol_shape, device="cuda")
                tigre.tigre_cgls(G.handle, b, x, 3)
                G.fdk(b)
        assert e.value.status == tigre.TIGRE_ERR_OOM
        gc.collect()
        torch.cuda.synchronize()
        assert not live
    finally:
        tigre.tigre_set_allocator(None, None)
    with tigre.Geometry(geo, ang) as G:
        assert torch.isfinite(G.forward(vol)).all()
