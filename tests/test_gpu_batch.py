"""Batched CGLS: several problems on one geometry handle iterated together,
one forward and one backprojection launch per iteration for the whole batch.
Every member's volume and residual history must be the single-problem
CGLS's bit for bit (same kernels per ray and per voxel, same fixed-order
reductions), in eager execution and in graph replay."""
import numpy as np
import pytest
import torch

from paper_1905_03748_gb300 import synth

pytestmark = pytest.mark.gpu


def ragged():
    geo = synth.geometry((37, 29, 21), (1.0, 0.9, 1.1), (53, 27), (1.05, 0.95), dso=300.0,
                         dsd=450.0, off_origin=(0.5, -0.3, 0.2), off_det=(1.3, -0.7))
    ang = np.sort(np.random.default_rng(4).uniform(0, 2 * np.pi, 23))
    return geo, ang


def head64():
    return synth.workload("small_64")


def alone(tigre, G, b, x0, n, x0_zero):
    x = x0.clone()
    st = tigre.tigre_cgls_begin(G.handle, b, x, n_iter_hint=n, x0_zero=x0_zero)
    tigre.tigre_cgls_iterate(st, n)
    h = tigre.tigre_cgls_history(st, n)
    tigre.tigre_cgls_end(st)
    torch.cuda.synchronize()
    return x, h


@pytest.mark.parametrize("which", ["ragged", "head64"])
@pytest.mark.parametrize("dtype,graph,x0_zero", [(torch.float32, False, True),
                                                 (torch.float32, True, True),
                                                 (torch.float32, True, False),
                                                 (torch.bfloat16, True, True)])
def test_each_member_equals_its_problem_alone(tigre, which, dtype, graph, x0_zero):
    geo, ang = ragged() if which == "ragged" else head64()
    nz, ny, nx = geo["n_voxel"][2], geo["n_voxel"][1], geo["n_voxel"][0]
    n_iter, B = 5, 3
    with tigre.Geometry(geo, ang) as G:
        bs, x0s = [], []
        for i in range(B):
            vol = torch.from_numpy(synth.random_volume((nz, ny, nx), seed=10 + i)).cuda()
            bs.append(G.forward(vol).to(dtype))
            x0s.append(torch.from_numpy(0.1 * synth.random_volume((nz, ny, nx), seed=20 + i))
                       .cuda().to(dtype))
        ref = [alone(tigre, G, bs[i], x0s[i], n_iter, x0_zero) for i in range(B)]
        s = torch.cuda.Stream()
        torch.cuda.synchronize()
        with torch.cuda.stream(s):
            xs = [x.clone() for x in x0s]
            st = tigre.tigre_cgls_batch_begin(G.handle, bs, xs, n_iter_hint=n_iter, stream=s,
                                              graph=graph, x0_zero=x0_zero)
            tigre.tigre_cgls_batch_iterate(st, 2)
            tigre.tigre_cgls_batch_iterate(st, n_iter - 2)
            hs = [tigre.tigre_cgls_batch_history(st, i, n_iter) for i in range(B)]
            tigre.tigre_cgls_batch_end(st)
            torch.cuda.synchronize()
    for i in range(B):
        assert torch.equal(xs[i], ref[i][0]), i
        np.testing.assert_array_equal(hs[i], ref[i][1])
    assert not torch.equal(xs[0], xs[1])


def test_a_batch_of_one_is_the_single_problem(tigre):
    geo, ang = ragged()
    with tigre.Geometry(geo, ang) as G:
        vol = torch.from_numpy(synth.random_volume((21, 29, 37), seed=3)).cuda()
        b = G.forward(vol)
        x_ref, h_ref = alone(tigre, G, b, torch.zeros_like(vol), 4, True)
        x = torch.full_like(vol, 5.0)
        st = tigre.tigre_cgls_batch_begin(G.handle, [b], [x], x0_zero=True)
        tigre.tigre_cgls_batch_iterate(st, 4)
        h = tigre.tigre_cgls_batch_history(st, 0, 4)
        tigre.tigre_cgls_batch_end(st)
        torch.cuda.synchronize()
    assert torch.equal(x, x_ref)
    np.testing.assert_array_equal(h, h_ref)


def test_batch_refusals(tigre):
    geo, ang = ragged()
    with tigre.Geometry(geo, ang) as G:
        b = torch.zeros(G.proj_shape, device="cuda")
        x = torch.zeros(G.vol_shape, device="cuda")
        with pytest.raises(tigre.TigreError) as e:
            tigre.tigre_cgls_batch_begin(G.handle, [b, b], [x, x.clone()], bp_weight="adjoint")
        assert e.value.status == tigre.TIGRE_ERR_UNSUPPORTED
        with pytest.raises(TypeError):
            tigre.tigre_cgls_batch_begin(G.handle, [b, b.bfloat16()], [x, x.bfloat16()])
        with pytest.raises(ValueError):
            tigre.tigre_cgls_batch_begin(G.handle, [b], [x, x])
        st = tigre.tigre_cgls_batch_begin(G.handle, [b, b], [x, x.clone()])
        try:
            with pytest.raises(tigre.TigreError):
                tigre.tigre_cgls_batch_history(st, 2, 0)  # no member 2
            with pytest.raises(tigre.TigreError):
                tigre.tigre_cgls_batch_history(st, 0, 1)  # no iteration done yet
        finally:
            tigre.tigre_cgls_batch_end(st)
