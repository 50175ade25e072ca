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


def case_volume_heavy():
    """A volume much larger than its projections (7 angles of a small
    detector): the regime where placement 1 (volume vectors in host memory,
    projections on the device) needs less device memory than placement 2."""
    geo = synth.geometry((61, 53, 47), (1.0, 0.9, 1.1), (23, 15), (1.6, 1.5), dso=300.0,
                         dsd=450.0, off_origin=(0.5, -0.3, 0.2), off_det=(1.3, -0.7))
    ang = np.sort(np.random.default_rng(4).uniform(0, 2 * np.pi, 7))
    vol = synth.random_volume((47, 53, 61), seed=6)
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


@pytest.mark.parametrize("brick", [5, 16])
def test_forward_ooc_in_xy_bricks_equals_in_core(tigre, brick):
    """Slabs cut into x-y bricks (many, with short last bricks): every sample
    is counted in exactly one brick, so the sums equal the in-core ones up to
    FP32 summation order; the per-angle column culling drops no ray."""
    geo, ang, vol = case()
    with tigre.Geometry(geo, ang) as G:
        ref = G.forward(torch.from_numpy(vol).cuda())
        tigre.tigre_geometry_set_brick(G.handle, brick)
        for path in (tigre.FWD_QUAD, tigre.FWD_QUAD_PAIR):
            tigre.tigre_geometry_set_forward_path(G.handle, path)
            out = torch.empty_like(ref)
            tigre.tigre_forward_ooc(G.handle, torch.from_numpy(vol.copy()), out, 0, len(ang),
                                    slab_planes=6)
            assert torch.isfinite(out).all()
            assert rel(out.cpu().numpy(), ref.cpu().numpy()) < 1e-6


def test_forward_ooc_paired_samples_bitwise(tigre):
    """The slab projection taking samples two at a time adds the same samples
    in the same order as the one-at-a-time kernel."""
    geo, ang, vol = case()
    outs = []
    with tigre.Geometry(geo, ang) as G:
        for path in (tigre.FWD_QUAD, tigre.FWD_QUAD_PAIR):
            tigre.tigre_geometry_set_forward_path(G.handle, path)
            out = torch.empty(G.proj_shape, device="cuda")
            tigre.tigre_forward_ooc(G.handle, torch.from_numpy(vol.copy()), out, 0, len(ang),
                                    slab_planes=4)
            outs.append(out)
    assert torch.isfinite(outs[0]).all()
    assert torch.equal(outs[0], outs[1])


@pytest.mark.parametrize("brick", [0, 16])
@pytest.mark.parametrize("a0,count", [(0, 19), (3, 11)])
def test_forward_ooc_angle_pairs_bitwise(tigre, brick, a0, count):
    """Slab projections with warps of two neighbouring angles (the full
    range's group table, or a partial range's own) add the same samples in
    the same order as one angle per warp, x-y bricks included."""
    geo, ang, vol = case()
    outs = []
    with tigre.Geometry(geo, ang) as G:
        if brick:
            tigre.tigre_geometry_set_brick(G.handle, brick)
        for path in (tigre.FWD_QUAD, tigre.FWD_QUAD_ANGLES2):
            tigre.tigre_geometry_set_forward_path(G.handle, path)
            out = torch.zeros((count, geo["n_det"][1], geo["n_det"][0]), device="cuda")
            tigre.tigre_forward_ooc(G.handle, torch.from_numpy(vol.copy()), out, a0, count,
                                    slab_planes=5)
            outs.append(out)
        ref = G.forward(torch.from_numpy(vol).cuda(), angle_begin=a0, angle_count=count)
        assert tigre.tigre_geometry_error_flags(G.handle) == 0
    assert torch.isfinite(outs[1]).all()
    assert torch.equal(outs[0], outs[1])
    assert rel(outs[1].cpu().numpy(), ref.cpu().numpy()) < 1e-6


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


@pytest.mark.parametrize("n_ang", [4, 16, 21])
@pytest.mark.parametrize("slab", [5, 16, 23])
@pytest.mark.parametrize("weight", ["matched", "fdk"])
def test_backward_ooc_quad_quarters(tigre, n_ang, slab, weight):
    """Slab backprojections build quad bands a quarter of the angles at a
    time (angle counts that fill the band buffer exactly and ones that leave
    a short last quarter; slab thicknesses that are not multiples of the
    voxels per thread): the same sums as in-core up to FP32 order."""
    geo, _, vol = case()
    ang = np.sort(np.random.default_rng(11).uniform(0, 2 * np.pi, n_ang))
    y = torch.from_numpy(np.random.default_rng(12).random(
        (n_ang, geo["n_det"][1], geo["n_det"][0])).astype(np.float32)).cuda()
    with tigre.Geometry(geo, ang) as G:
        ref = G.backward(y, weight=weight).cpu()
        out = torch.zeros(G.vol_shape).pin_memory()
        tigre.tigre_backward_ooc(G.handle, y, out, 0, n_ang, weight=weight, slab_planes=slab)
        assert tigre.tigre_geometry_error_flags(G.handle) == 0
    assert torch.isfinite(out).all()
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


def budgets_by_plan(tigre, G):
    """Device budgets that give each (placement, slab planes) plan, smallest
    budget per plan, scanning 64 KiB .. 64 MiB."""
    plans = {}
    b = 64 << 10
    while b < (64 << 20):
        try:
            plans.setdefault(tigre.tigre_cgls_ooc_plan(G.handle, b), b)
        except tigre.TigreError:
            pass
        b = int(b * 1.03) + 1
    return plans


def test_ooc_plan_orders_placements(tigre):
    geo, ang, _ = case_volume_heavy()
    with tigre.Geometry(geo, ang) as G:
        plans = budgets_by_plan(tigre, G)
        with pytest.raises(tigre.TigreError):
            tigre.tigre_cgls_ooc_plan(G.handle, 1024)
        assert tigre.tigre_cgls_ooc_plan(G.handle, 0) == (2, 47)
    ones = sorted(b for (pl, _), b in plans.items() if pl == 1)
    twos = sorted(b for (pl, _), b in plans.items() if pl == 2)
    assert ones and twos and max(ones) < min(twos)
    # thicker slabs need more budget
    for pl in (1, 2):
        got = sorted((b, sl) for (p_, sl), b in plans.items() if p_ == pl)
        assert [sl for _, sl in got] == sorted(sl for _, sl in got)


def pick(plans, placement, max_slab):
    cands = [(sl, b) for (pl, sl), b in plans.items() if pl == placement and sl <= max_slab]
    assert cands, (placement, max_slab, plans)
    return max(cands)


@pytest.mark.parametrize("placement,max_slab,x0", [(0, 0, False), (2, 1, False), (2, 4, True),
                                                   (1, 3, False), (1, 3, True)])
def test_cgls_out_of_core_equals_in_core(tigre, placement, max_slab, x0):
    """Placement 2 (x, r, q on the device, direction streamed through the
    host buffer, s recomputed) and placement 1 (x, p, s in host memory), with
    slabs forced thin so that many slabs, the three-buffer ring and a short
    last slab are exercised; same iterates and residuals as the in-core CGLS
    up to FP32 summation order."""
    geo, ang, vol = case_volume_heavy() if placement == 1 else case()
    b = oracle.forward(geo, ang, vol).astype(np.float32)
    start = (0.3 * synth.random_volume(vol.shape, seed=9)).astype(np.float32) if x0 else \
        np.zeros(vol.shape, np.float32)
    with tigre.Geometry(geo, ang) as G:
        budget = 0
        if placement:
            slab, budget = pick(budgets_by_plan(tigre, G), placement, max_slab)
            assert tigre.tigre_cgls_ooc_plan(G.handle, budget) == (placement, slab)
        xd = torch.from_numpy(start.copy()).cuda()
        hd = tigre.tigre_cgls(G.handle, torch.from_numpy(b).cuda(), xd, 6)
        xh = torch.from_numpy(start.copy())
        hh = tigre.tigre_cgls(G.handle, torch.from_numpy(b), xh, 6, out_of_core=True,
                              device_budget_bytes=budget)
    np.testing.assert_allclose(hh, hd, rtol=1e-5)
    assert rel(xh.numpy(), xd.cpu().numpy()) < 1e-5


@pytest.mark.parametrize("n_iter", [0, 1, 2])
def test_cgls_streamed_direction_short_runs(tigre, n_iter):
    """0 iterations leave x as given; 1 iteration is the first sweep plus the
    x-only pass; 2 adds one full norm and update sweep."""
    geo, ang, vol = case()
    b = oracle.forward(geo, ang, vol).astype(np.float32)
    with tigre.Geometry(geo, ang) as G:
        slab, budget = pick(budgets_by_plan(tigre, G), 2, 5)
        xd = torch.zeros(G.vol_shape, device="cuda")
        hd = tigre.tigre_cgls(G.handle, torch.from_numpy(b).cuda(), xd, n_iter)
        xh = torch.zeros(G.vol_shape)
        hh = tigre.tigre_cgls(G.handle, torch.from_numpy(b), xh, n_iter, out_of_core=True,
                              device_budget_bytes=budget)
    np.testing.assert_allclose(hh, hd, rtol=1e-5)
    if n_iter == 0:
        assert not xh.any()
    else:
        assert rel(xh.numpy(), xd.cpu().numpy()) < 1e-5


@pytest.mark.parametrize("slab,depth,steps", [(6, 2, 5), (4, 4, 4), (23, 3, 3), (1, 1, 2)])
def test_tv_out_of_core_matches_split_oracle(tigre, slab, depth, steps):
    """Split TV on a host volume: the same rounds, buffers and per-slab norms
    as the oracle's split (short last slab, buffers at both ends)."""
    vol = synth.random_volume((23, 29, 37), seed=22)
    ref = oracle.tv_steps_split(vol, steps, 0.02, 1e-8, slab=slab, depth=depth)
    h = torch.from_numpy(vol.copy())
    tigre.tigre_tv_step_ooc(h, steps, 0.02, 1e-8, slab_planes=slab, halo_depth=depth)
    assert rel(h.numpy(), ref) < 1e-5


def test_tv_out_of_core_one_slab_is_the_in_core_step(tigre):
    vol = synth.random_volume((11, 13, 17), seed=23)
    d = torch.from_numpy(vol.copy()).cuda()
    tigre.tigre_tv_step(d, 4, 0.03, 1e-8)
    h = torch.from_numpy(vol.copy())
    tigre.tigre_tv_step_ooc(h, 4, 0.03, 1e-8, slab_planes=0, halo_depth=2)
    assert torch.equal(h, d.cpu())


def test_tv_out_of_core_rejects_a_buffer_deeper_than_the_slab(tigre):
    h = torch.zeros((8, 4, 4))
    with pytest.raises(tigre.TigreError):
        tigre.tigre_tv_step_ooc(h, 2, 0.1, slab_planes=2, halo_depth=3)


def test_plan_from_a_description_equals_the_handle_plan(tigre):
    """The host-only planner and the handle's planner take the same decision."""
    geo, ang = synth.workload("cgls_512")
    with tigre.Geometry(geo, ang) as G:
        for budget in (40 * 10 ** 9, 2 * 10 ** 9, 1_500_000_000, 1_300_000_000):
            assert (tigre.tigre_cgls_ooc_plan(G.handle, budget)
                    == tigre.tigre_cgls_ooc_plan_desc(geo, ang, budget))
