"""CUDA-graph CGLS and the continuous-batching server: every request's result
is the same alone and in the mix (bitwise: each request has its own buffers
and the kernels are deterministic)."""
import numpy as np
import pytest
import torch

from paper_1905_03748_gb300 import synth

pytestmark = pytest.mark.gpu


def make_request(i, rng, n=None):
    n = n or int(rng.choice([24, 32, 40]))
    na = int(rng.choice([18, 30]))
    geo = synth.cube_geometry(n, int(1.5 * n) + (i % 3), fov_mm=64.0)
    ang = synth.angles(na) + 0.01 * i
    vol = synth.voxelize(synth.random_ellipsoids(n, 64.0 / n, 5, seed=100 + i, r_vox=(60, 200)),
                         geo["n_voxel"], geo["d_voxel"])
    return geo, ang, vol


def projections(tigre, geo, ang, vol):
    with tigre.Geometry(geo, ang) as G:
        return G.forward(torch.from_numpy(vol).cuda()).cpu()


@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16])
def test_graph_replay_equals_eager_iterations(tigre, dtype):
    rng = np.random.default_rng(0)
    geo, ang, vol = make_request(0, rng, n=32)
    b = projections(tigre, geo, ang, vol).cuda().to(dtype)
    out = {}
    for graph in (False, True):
        s = torch.cuda.Stream()
        with torch.cuda.stream(s), tigre.Geometry(geo, ang) as G:
            x = torch.zeros(G.vol_shape, device="cuda", dtype=dtype)
            st = tigre.tigre_cgls_begin(G.handle, b, x, n_iter_hint=4, stream=s, graph=graph)
            tigre.tigre_cgls_iterate(st, 1)   # odd first: exercises both graph parities
            tigre.tigre_cgls_iterate(st, 6)
            h = tigre.tigre_cgls_history(st, 7)
            tigre.tigre_cgls_end(st)
            torch.cuda.synchronize()
            out[graph] = (x.float().cpu(), h)
    assert torch.equal(out[False][0], out[True][0])
    np.testing.assert_array_equal(out[False][1], out[True][1])
    assert np.all(np.diff(out[True][1]) < 0)


@pytest.mark.parametrize("budget_mb", [None, 64])
def test_each_request_same_alone_and_in_the_mix(tigre, budget_mb):
    from paper_1905_03748_gb300 import serving
    rng = np.random.default_rng(1)
    reqs = []
    for i in range(6):
        geo, ang, vol = make_request(i, rng)
        b = projections(tigre, geo, ang, vol)
        if i % 2:  # every other request is served with BF16 storage
            b = b.to(torch.bfloat16)
        reqs.append(serving.Request(i, geo, ang, b.pin_memory(), n_iter=5 + (i % 3),
                                    arrival=0.002 * i))
    alone = {r.rid: r for r in serving.run_plain(reqs, realtime=False)}
    budget = None if budget_mb is None else budget_mb << 20
    server = serving.Server(max_slots=4, hbm_budget=budget, graph=True, iters_per_tick=2)
    mixed = server.run(reqs, realtime=True)
    assert sorted(r.rid for r in mixed) == list(range(6))
    for r in mixed:
        assert torch.equal(r.x, alone[r.rid].x), r.rid
        np.testing.assert_array_equal(r.resid, alone[r.rid].resid)
    stats = serving.latency_stats(mixed)
    assert stats["p99_s"] >= stats["p50_s"] > 0


def test_batched_groups_same_alone_and_in_the_mix(tigre):
    """Requests that share geometry, angles, storage type and iteration count
    are served as batched CGLS groups (one forward and one backprojection
    launch per iteration for the group); each result is bitwise its problem
    solved alone."""
    from paper_1905_03748_gb300 import serving
    keys = [(synth.cube_geometry(32, 48, fov_mm=64.0), synth.angles(30)),
            (synth.cube_geometry(24, 40, fov_mm=64.0), synth.angles(18) + 0.1)]
    reqs = []
    for i in range(8):
        geo, ang = keys[i % 2]
        n = geo["n_voxel"][0]
        vol = synth.voxelize(synth.random_ellipsoids(n, 64.0 / n, 5, seed=200 + i,
                                                     r_vox=(60, 200)),
                             geo["n_voxel"], geo["d_voxel"])
        b = projections(tigre, geo, ang, vol)
        if i == 5:  # a BF16 request: a key of its own
            b = b.to(torch.bfloat16)
        reqs.append(serving.Request(i, geo, ang, b.pin_memory(), n_iter=6, arrival=0.0))
    alone = {r.rid: r for r in serving.run_plain(reqs, realtime=False)}
    server = serving.Server(max_slots=8, graph=True, iters_per_tick=2, max_batch=3)
    mixed = server.run(reqs, realtime=False)
    assert sorted(r.rid for r in mixed) == list(range(8))
    assert max(len(g) for g in server.groups) == 3 and [5] in server.groups
    for r in mixed:
        assert torch.equal(r.x, alone[r.rid].x), r.rid
        np.testing.assert_array_equal(r.resid, alone[r.rid].resid)
