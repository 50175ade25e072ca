"""tigre_tv_step_noalloc: the TV step for callers that cannot allocate device
memory while they run (a real-time loop that reserved its memory at
start-up, or a process whose memory another allocator holds).  It must give
the same result as tigre_tv_step, call after call, through the C ABI.

This file is collected last on purpose (name order), so a run that stops at
its first failure has already run every other test.
"""
import gc

import numpy as np
import pytest
import torch

from paper_1905_03748_gb300 import synth

pytestmark = pytest.mark.gpu
TOL = 1e-4  # the relative-L2 tolerance of the FP32 parity tests


def rel(a, b):
    a = a.double().cpu().numpy()
    b = b.double().cpu().numpy()
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_noalloc_tv_step_matches_tv_step_on_two_calls(tigre):
    vol = synth.voxelize(synth.random_ellipsoids(40, 1.0, 8, seed=3, r_vox=(60, 160)),
                         (40, 36, 28), (1.0, 1.0, 1.0))
    vol = vol + 0.01 * synth.random_volume(vol.shape, seed=4)
    ref = torch.from_numpy(vol).cuda()
    out = ref.clone()
    for _ in range(2):  # the second call reuses the scratch the first one left
        tigre.tigre_tv_step(ref, 3, 0.5, 1e-8)
        tigre.tigre_tv_step_noalloc(out, 3, 0.5, 1e-8)
        torch.cuda.synchronize()
        assert torch.isfinite(out).all()
        assert rel(out, ref) < TOL
    assert not torch.equal(out, torch.from_numpy(vol).cuda())  # the steps did move x


def test_noalloc_tv_step_rejects_volumes_beyond_its_scratch(tigre):
    big = torch.zeros((161, 160, 164), device="cuda")  # 4,224,640 voxels > 4,194,304
    with pytest.raises(tigre.TigreError, match="scratch"):
        tigre.tigre_tv_step_noalloc(big, 1, 0.1, 1e-8)


def test_noalloc_tv_step_calls_no_allocator(tigre):
    """After the set-up call (n_steps = 0) on this device, two calls go
    through with an allocator that refuses everything and counts its calls:
    it is never called.  tigre_tv_step, which allocates its scratch per
    call, fails under the same allocator."""
    vol = synth.random_volume((24, 30, 34), seed=6)
    x = torch.from_numpy(vol).cuda()
    ref = x.clone()
    tigre.tigre_tv_step_noalloc(x, 0, 0.5, 1e-8)  # the per-device set-up
    torch.cuda.synchronize()
    calls = {"alloc": 0, "free": 0}

    def alloc(nbytes, stream):
        calls["alloc"] += 1
        return 0  # refuse

    def free(ptr, stream):
        calls["free"] += 1

    gc.collect()  # handles left to the garbage collector by earlier tests
    tigre.tigre_set_allocator(alloc, free)
    try:
        for _ in range(2):
            tigre.tigre_tv_step_noalloc(x, 3, 0.5, 1e-8)
        torch.cuda.synchronize()
        seen = dict(calls)
        with pytest.raises(tigre.TigreError) as err:
            tigre.tigre_tv_step(ref.clone(), 3, 0.5, 1e-8)
        assert err.value.status == tigre.TIGRE_ERR_OOM
    finally:
        torch.cuda.synchronize()
        tigre.tigre_set_allocator(None, None)
    assert seen == {"alloc": 0, "free": 0}
    for _ in range(2):
        tigre.tigre_tv_step(ref, 3, 0.5, 1e-8)
    torch.cuda.synchronize()
    assert rel(x, ref) < TOL
