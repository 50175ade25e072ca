"""GPU parity of the ray-voxel intersection (Siddon) projector and its exact
transpose against the FP64 oracle, through the C ABI.

Tolerance 1e-4 relative L2 (FP32), as for the interpolated projector; the
512^3 x 360 workload is checked on sampled rays.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1905_03748_gb300 import synth

pytestmark = pytest.mark.gpu
TOL = 1e-4


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def ragged_case():
    geo = synth.geometry((37, 29, 21), (1.0, 0.9, 1.1), (53, 27), (1.05, 0.95), dso=300.0,
                         dsd=450.0, off_origin=(0.5, -0.3, 0.2), off_det=(1.3, -0.7))
    ang = np.sort(np.random.default_rng(4).uniform(0, 2 * np.pi, 23))
    return geo, ang, synth.random_volume((21, 29, 37), seed=5)


def small_case():
    geo, ang = synth.workload("small_64")
    return geo, ang, synth.phantom("head10", 64, 1.0)


def axis_case(off_det=(0.25, 0.25)):
    """Angles on the axes and the diagonals: axis-parallel rays (direction
    components that are zero or nearly so) and rays through voxel edges.  The
    default quarter-pixel detector shift keeps every ray off the voxel faces;
    off_det=(0, 0) puts some rays exactly on faces."""
    geo = synth.geometry(16, 1.0, (33, 17), 1.0, dso=100.0, dsd=150.0, off_det=off_det)
    ang = np.arange(8) * (np.pi / 4)
    return geo, ang, synth.random_volume((16, 16, 16), seed=6)


CASES = {"ragged": ragged_case, "small_64": small_case, "axes": axis_case}


@pytest.fixture(scope="module", params=list(CASES))
def case(request):
    return CASES[request.param]()


def test_siddon_forward_matches_oracle(tigre, case):
    geo, ang, vol = case
    with tigre.Geometry(geo, ang) as G:
        tigre.tigre_geometry_set_projector(G.handle, "siddon")
        p = G.forward(torch.from_numpy(vol).cuda()).cpu().numpy()
    ref = oracle.siddon_forward(geo, ang, vol)
    assert np.isfinite(p).all()
    assert rel(p, ref) < TOL


def test_siddon_rays_on_voxel_faces_take_one_side(tigre):
    """A ray lying exactly on a face between two voxels has no unique Siddon
    value (the volume jumps there).  In FP64 the oracle's ray on such a face
    is tilted by the rounding of cos/sin and crosses it part-way; the GPU's
    FP32 direction is exactly axis-parallel and stays on one side.  Each GPU
    value must equal the oracle's value or that of the ray nudged off the
    face to one side (detector shifted by +-eps); off the faces all of these
    coincide."""
    geo, ang, vol = axis_case(off_det=(0.0, 0.0))
    with tigre.Geometry(geo, ang) as G:
        tigre.tigre_geometry_set_projector(G.handle, "siddon")
        got = G.forward(torch.from_numpy(vol).cuda()).cpu().numpy().astype(np.float64)
    eps = 1e-5
    cands = [oracle.siddon_forward(geo, ang, vol)]
    cands += [oracle.siddon_forward(dict(geo, off_det=(du, dv)), ang, vol)
              for du in (-eps, eps) for dv in (-eps, eps)]
    cands = np.array(cands)
    tol = 1e-4 * np.abs(cands).max()
    ok = np.any(np.abs(cands - got[None]) <= tol, axis=0)
    assert ok.all(), np.argwhere(~ok)[:5]
    assert (cands.max(0) - cands.min(0)).max() > 0.1  # the geometry does put rays on faces


def test_siddon_forward_subrange_and_dtypes(tigre):
    geo, ang, vol = ragged_case()
    ref = oracle.siddon_forward(geo, ang[5:12], vol)
    with tigre.Geometry(geo, ang) as G:
        tigre.tigre_geometry_set_projector(G.handle, tigre.PROJ_SIDDON)
        v = torch.from_numpy(vol).cuda()
        sub = G.forward(v, angle_begin=5, angle_count=7).cpu().numpy()
        half = G.forward(v.to(torch.bfloat16), dtype=torch.float32).cpu().numpy()
    assert rel(sub, ref) < TOL
    # BF16 storage: the input is rounded to 8 bits of mantissa
    assert rel(half[5:12], ref) < 1e-2


def test_siddon_exact_adjoint_matches_oracle_and_dot_test(tigre):
    geo, ang, _ = ragged_case()
    rng = np.random.default_rng(9)
    y = rng.random((len(ang), 27, 53)).astype(np.float32)
    x = rng.random((21, 29, 37)).astype(np.float32)
    with tigre.Geometry(geo, ang) as G:
        tigre.tigre_geometry_set_projector(G.handle, "siddon")
        aty = G.backward(torch.from_numpy(y).cuda(), weight="adjoint").cpu().numpy()
        ax = G.forward(torch.from_numpy(x).cuda()).cpu().numpy()
    assert rel(aty, oracle.siddon_adjoint(geo, ang, y)) < TOL
    lhs = float(np.sum(ax.astype(np.float64) * y))
    rhs = float(np.sum(x.astype(np.float64) * aty))
    assert abs(lhs - rhs) <= 1e-5 * abs(lhs)


def test_siddon_cgls_matches_oracle(tigre):
    geo, ang, vol = ragged_case()
    b = oracle.siddon_forward(geo, ang, vol)
    x_ref, h_ref = oracle.cgls(geo, ang, b, 8, bp="adjoint", projector="siddon")
    with tigre.Geometry(geo, ang) as G:
        tigre.tigre_geometry_set_projector(G.handle, "siddon")
        x = torch.zeros(G.vol_shape, device="cuda")
        h = tigre.tigre_cgls(G.handle, torch.from_numpy(b.astype(np.float32)).cuda(), x, 8,
                             bp_weight="adjoint")
    np.testing.assert_allclose(h, h_ref, rtol=1e-4)
    assert rel(x.cpu().numpy(), x_ref) < 1e-3


def test_siddon_out_of_core_is_refused(tigre):
    geo, ang, vol = ragged_case()
    with tigre.Geometry(geo, ang) as G:
        tigre.tigre_geometry_set_projector(G.handle, "siddon")
        out = torch.empty(G.proj_shape, device="cuda")
        with pytest.raises(tigre.TigreError):
            tigre.tigre_forward_ooc(G.handle, torch.from_numpy(vol.copy()), out, 0, len(ang),
                                    slab_planes=4)


def test_siddon_full_size_sampled_rays(tigre):
    """512^3 x 360 (the benchmark workload): 3000 sampled rays one by one."""
    geo, ang = synth.workload("cgls_512")
    vol = synth.phantom("ellipsoids50", 512, 0.5)
    rays = synth.random_rays(len(ang), 512, 512, 3000, seed=21)
    ref = oracle.siddon_forward_rays(geo, ang, vol, rays)
    with tigre.Geometry(geo, ang) as G:
        tigre.tigre_geometry_set_projector(G.handle, "siddon")
        p = G.forward(torch.from_numpy(vol).cuda())
        got = p[rays[:, 0], rays[:, 1], rays[:, 2]].cpu().numpy()
    assert rel(got, ref) < TOL
