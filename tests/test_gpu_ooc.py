"""Out-of-core operators (Alg. 1 / Alg. 2 on one GPU) against the in-core
ones and the oracle, with slabs and angle chunks forced small so that many
slabs (and a short last slab) are exercised."""
import numpy as np
import pytest
import torch

import oracle
from paper_1905_03748_gb300 import synth

pytestmark = pytest.mark.gpu


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def case():
    geo = synth.geometry((37, 29, 23), (1.0, 0.9, 1.1), (53, 31), (1.05, 0.95), dso=300.0,
                         dsd=450.0, off_origin=(0.5, -0.3, 0.2), off_det=(1.3, -0.7))
    ang = np.sort(np.random.default_rng(4).uniform(0, 2 * np.pi, 19))
    vol = synth.random_volume((23, 29, 37), seed=5)
    return geo, ang, vol


@pytest.mark.parametrize("slab", [1, 3, 7, 23])
@pytest.mark.parametrize("pinned", [True, False])
def test_forward_ooc_equals_in_core(tigre, slab, pinned):
    geo, ang, vol = case()
    with tigre.Geometry(geo, ang) as G:
        ref = G.forward(torch.from_numpy(vol).cuda())
        vh = torch.from_numpy(vol.copy())
        if pinned:
            vh = vh.pin_memory()
        out = torch.empty_like(ref)
        tigre.tigre_forward_ooc(G.handle, vh, out, 0, len(ang), slab_planes=slab)
    assert torch.isfinite(out).all()
    assert rel(out.cpu().numpy(), ref.cpu().numpy()) < 1e-6
    if slab == 3 and pinned:
        assert rel(out.cpu().numpy(), oracle.forward(geo, ang, vol)) < 1e-4


@pytest.mark.parametrize("slab", [1, 5, 23])
@pytest.mark.parametrize("weight", ["matched", "fdk"])
def test_backward_ooc_device_projections(tigre, slab, weight):
    """Same sums as in-core; a slab launch computes a voxel's z from its own
    first plane, so the last bits may differ (1e-6)."""
    geo, ang, vol = case()
    y = torch.from_numpy(np.random.default_rng(7).random(
        (len(ang), geo["n_det"][1], geo["n_det"][0])).astype(np.float32)).cuda()
    with tigre.Geometry(geo, ang) as G:
        ref = G.backward(y, weight=weight).cpu()
        out = torch.zeros(G.vol_shape).pin_memory()
        tigre.tigre_backward_ooc(G.handle, y, out, 0, len(ang), weight=weight, slab_planes=slab)
    assert rel(out.numpy(), ref.numpy()) < 1e-6


@pytest.mark.parametrize("chunk", [1, 4, 19])
def test_backward_ooc_host_projections_in_chunks(tigre, chunk):
    geo, ang, vol = case()
    y_np = np.random.default_rng(8).random((len(ang), geo["n_det"][1], geo["n_det"][0]))
    y_np = y_np.astype(np.float32)
    with tigre.Geometry(geo, ang) as G:
        ref = G.backward(torch.from_numpy(y_np).cuda()).cpu().numpy()
        out = torch.zeros(G.vol_shape)
        tigre.tigre_backward_ooc(G.handle, torch.from_numpy(y_np), out, 0, len(ang),
                                 slab_planes=4, angle_chunk=chunk)
    assert rel(out.numpy(), ref) < 1e-6
    if chunk == 4:
        assert rel(out.numpy(), oracle.backward(geo, ang, y_np)) < 1e-4


@pytest.mark.parametrize("budget_mb", [0, 2])
def test_cgls_out_of_core_equals_in_core(tigre, budget_mb):
    """Volume vectors in host memory, streamed in z-slabs (2 MB budget: slabs
    of a few planes); same iterates and residuals as the in-core CGLS up to
    FP32 summation order."""
    geo, ang, vol = case()
    b = oracle.forward(geo, ang, vol).astype(np.float32)
    with tigre.Geometry(geo, ang) as G:
        xd = torch.zeros(G.vol_shape, device="cuda")
        hd = tigre.tigre_cgls(G.handle, torch.from_numpy(b).cuda(), xd, 6)
        xh = torch.zeros(G.vol_shape)
        hh = tigre.tigre_cgls(G.handle, torch.from_numpy(b), xh, 6, out_of_core=True,
                              device_budget_bytes=budget_mb << 20)
    np.testing.assert_allclose(hh, hd, rtol=1e-5)
    assert rel(xh.numpy(), xd.cpu().numpy()) < 1e-5
