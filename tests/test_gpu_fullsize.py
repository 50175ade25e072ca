"""Full-size parity on sampled outputs: the 512^3 x 360 workload in the
launch configuration the benchmark times, and the 1024^3 x 720 workload per
storage type.  The oracle evaluates each sampled ray / voxel on its own
(FP64); the measured errors are printed (run with -s to see them)."""
import numpy as np
import pytest
import torch

import oracle
from paper_1905_03748_gb300 import synth

pytestmark = pytest.mark.gpu


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def w512():
    geo, ang = synth.workload("cgls_512")
    x = synth.phantom("ellipsoids50", 512, 0.5, seed=2)
    return geo, ang, x


def test_512_forward_backward_adjoint_sampled(tigre, w512):
    geo, ang, x = w512
    rays = synth.random_rays(len(ang), 512, 512, 3000, seed=21)
    vox = synth.random_voxels(512, 512, 512, 3000, seed=22)
    with tigre.Geometry(geo, ang) as G:
        xt = torch.from_numpy(x).cuda()
        p = G.forward(xt)
        assert torch.isfinite(p).all()
        y = p.cpu().numpy()
        bm = G.backward(p, weight="matched")
        bf = G.backward(p, weight="fdk")
        ba = G.backward(p, weight="adjoint")
        assert tigre.tigre_geometry_error_flags(G.handle) == 0
    x64 = x.astype(np.float64)
    e_fwd = rel(y[rays[:, 0], rays[:, 1], rays[:, 2]], oracle.forward_rays(geo, ang, x64, rays))
    sel = lambda t: t[vox[:, 2], vox[:, 1], vox[:, 0]].cpu().numpy()  # noqa: E731
    e_bm = rel(sel(bm), oracle.backward_voxels(geo, ang, y, vox, oracle.BP_MATCHED))
    e_bf = rel(sel(bf), oracle.backward_voxels(geo, ang, y, vox, oracle.BP_FDK))
    vox_a = vox[:256]
    e_ba = rel(sel(ba)[:256], oracle.adjoint_voxels(geo, ang, y, vox_a))
    print(f"\n512^3x360 sampled rel err: forward {e_fwd:.2e}, matched BP {e_bm:.2e}, "
          f"FDK BP {e_bf:.2e}, exact adjoint {e_ba:.2e}")
    # One voxel's exact-adjoint value is a sum over individual samples, so
    # it is sensitive to a ray's sample count: one sample more or less moves
    # every sample of that ray.  The GPU counts them as the quadrature does
    # (FP32 set-up, FP64 where FP32 cannot decide), so the bound is the
    # operators' own.
    assert e_fwd < 1e-4 and e_bm < 1e-4 and e_bf < 1e-4 and e_ba < 1e-4


def test_512_sample_counts_equal_the_oracle_angle_by_angle(tigre, w512):
    """The number of quadrature samples of every ray, summed per angle, is
    the oracle's: K = max(1, ceil(len/step - 1e-9)) decided exactly, not
    within FP32 rounding (an integer result: compared exactly)."""
    geo, ang, _ = w512
    with tigre.Geometry(geo, ang) as G:
        dev = [tigre.tigre_forward_samples(G.handle, a, 1) for a in range(len(ang))]
    ref = [oracle.sample_count(geo, ang[a:a + 1]) for a in range(len(ang))]
    assert dev == ref


@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16, torch.float16])
def test_1024_storage_types_sampled(tigre, dtype):
    """Operators with the volume / projections stored in `dtype`: parity with
    the oracle on the storage-rounded inputs (1e-4), and the error the storage
    type adds against the oracle on the FP32 inputs (reported; bounded by
    the format's precision)."""
    geo, ang = synth.workload("mixed_1024")
    x = synth.voxelize(synth.random_ellipsoids(1024, 0.25, 50, seed=3), geo["n_voxel"],
                       geo["d_voxel"])
    rays = synth.random_rays(len(ang), 1024, 1024, 1500, seed=31)
    vox = synth.random_voxels(1024, 1024, 1024, 1500, seed=32)
    with tigre.Geometry(geo, ang) as G:
        xs = torch.from_numpy(x).cuda().to(dtype)
        p = G.forward(xs, dtype=torch.float32)
        ys = p.to(dtype)
        bp = G.backward(ys, weight="matched", dtype=torch.float32)
        p_s = p[rays[:, 0], rays[:, 1], rays[:, 2]].cpu().numpy()
        bp_s = bp[vox[:, 2], vox[:, 1], vox[:, 0]].cpu().numpy()
        x_round = xs.float().cpu().numpy().astype(np.float64)
        y_round = ys.float().cpu().numpy()
        y32 = p.cpu().numpy()
        del xs, p, ys, bp
    e_fwd = rel(p_s, oracle.forward_rays(geo, ang, x_round, rays))
    e_bp = rel(bp_s, oracle.backward_voxels(geo, ang, y_round, vox))
    f_fwd = rel(p_s, oracle.forward_rays(geo, ang, x.astype(np.float64), rays))
    f_bp = rel(bp_s, oracle.backward_voxels(geo, ang, y32, vox))
    print(f"\n1024^3x720 {dtype}: parity forward {e_fwd:.2e} BP {e_bp:.2e}; "
          f"storage error vs FP32-input oracle: forward {f_fwd:.2e} BP {f_bp:.2e}")
    assert e_fwd < 1e-4 and e_bp < 1e-4
    bound = {torch.float32: 1e-4, torch.bfloat16: 1e-2, torch.float16: 2e-3}[dtype]
    assert f_fwd < bound and f_bp < bound
