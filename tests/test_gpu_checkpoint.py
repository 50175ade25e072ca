"""Checkpoint / resume of the stepwise CGLS: a state saved after some
iterations (x, r, p, gamma) and resumed in a fresh state continues as the
uninterrupted iteration does -- bitwise with the matched backprojector (same
kernels, same inputs, fixed reduction order), to rounding with the exact
adjoint (its scatter sums with atomics, in no fixed order)."""
import numpy as np
import pytest
import torch

from paper_1905_03748_gb300 import synth

pytestmark = pytest.mark.gpu


def case():
    geo = synth.geometry((37, 29, 21), (1.0, 0.9, 1.1), (53, 27), (1.05, 0.95), dso=300.0,
                         dsd=450.0, off_origin=(0.5, -0.3, 0.2), off_det=(1.3, -0.7))
    ang = np.sort(np.random.default_rng(4).uniform(0, 2 * np.pi, 23))
    return geo, ang, synth.random_volume((21, 29, 37), seed=5)


@pytest.mark.parametrize("dtype,graph,bp", [(torch.float32, False, "matched"),
                                            (torch.float32, True, "matched"),
                                            (torch.bfloat16, False, "matched"),
                                            (torch.float32, False, "adjoint")])
def test_resume_continues(tigre, dtype, graph, bp):
    geo, ang, vol = case()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s), tigre.Geometry(geo, ang) as G:
        b = G.forward(torch.from_numpy(vol).cuda()).to(dtype)
        # uninterrupted: 3 + 4 iterations, checkpoint taken after the first 3
        x = torch.zeros(G.vol_shape, device="cuda", dtype=dtype)
        st = tigre.tigre_cgls_begin(G.handle, b, x, n_iter_hint=8, stream=s, graph=graph,
                                    bp_weight=bp)
        tigre.tigre_cgls_iterate(st, 3)
        r_host = torch.empty(G.proj_shape, dtype=dtype)
        p_host = torch.empty(G.vol_shape, dtype=dtype)
        gamma, done = tigre.tigre_cgls_save(st, r_host, p_host)
        x_ck = x.cpu()
        tigre.tigre_cgls_iterate(st, 4)
        h_ref = tigre.tigre_cgls_history(st, 7)
        tigre.tigre_cgls_end(st)
        torch.cuda.synchronize()
        x_ref = x.cpu()
        # resumed in a fresh state on a fresh handle (no workspace cached yet:
        # with graph=True the first replay is captured before any projection)
        x2 = x_ck.cuda()
        with tigre.Geometry(geo, ang) as G2:
            st2 = tigre.tigre_cgls_resume(G2.handle, b, x2, r_host, p_host, gamma,
                                          n_iter_hint=8, stream=s, graph=graph, bp_weight=bp)
            tigre.tigre_cgls_iterate(st2, 4)
            h2 = tigre.tigre_cgls_history(st2, 4)
            tigre.tigre_cgls_end(st2)
            torch.cuda.synchronize()
    assert done == 3 and gamma > 0 and np.isfinite(gamma)
    if bp == "matched":
        assert torch.equal(x2.cpu(), x_ref)
        np.testing.assert_array_equal(h2, h_ref[3:])
    else:
        d = (x2.cpu() - x_ref).double().norm() / x_ref.double().norm()
        assert float(d) < 1e-5
        np.testing.assert_allclose(h2, h_ref[3:], rtol=1e-5)
        assert np.all(np.diff(h_ref) < 0)  # exact adjoint: the residual norm decreases


@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16])
def test_graph_replay_from_a_zero_start_on_a_fresh_handle(tigre, dtype):
    """begin(graph=True, x0_zero=True) on a handle that has never projected:
    the zero start skips A x0, so the first projection of the run is the
    one captured into the graph.  The workspaces it needs are made when the
    state is, and the replayed iterations are the eager ones bit for bit."""
    geo, ang, vol = case()
    with tigre.Geometry(geo, ang) as G0:
        b = G0.forward(torch.from_numpy(vol).cuda()).to(dtype)
        x_ref = torch.zeros(G0.vol_shape, device="cuda", dtype=dtype)
        st = tigre.tigre_cgls_begin(G0.handle, b, x_ref, x0_zero=True)
        tigre.tigre_cgls_iterate(st, 5)
        h_ref = tigre.tigre_cgls_history(st, 5)
        tigre.tigre_cgls_end(st)
    s = torch.cuda.Stream()
    torch.cuda.synchronize()
    with torch.cuda.stream(s), tigre.Geometry(geo, ang) as G:
        x = torch.full(G.vol_shape, 3.0, device="cuda", dtype=dtype)
        st = tigre.tigre_cgls_begin(G.handle, b, x, stream=s, graph=True, x0_zero=True)
        tigre.tigre_cgls_iterate(st, 5)  # two captured pairs, then one eager step
        h = tigre.tigre_cgls_history(st, 5)
        tigre.tigre_cgls_end(st)
        torch.cuda.synchronize()
    assert torch.equal(x, x_ref)
    np.testing.assert_array_equal(h, h_ref)


def test_graph_replay_with_in_core_bricks_on_a_fresh_handle(tigre):
    """With x-y bricks forced small the automatic projection marches bricks
    (a zeroing memset, then one launch per brick): CGLS iterations captured
    into a graph on a fresh handle equal the eager ones bit for bit."""
    geo, ang, vol = case()
    v = torch.from_numpy(vol).cuda()
    with tigre.Geometry(geo, ang) as G0:
        tigre.tigre_geometry_set_brick(G0.handle, 16)
        b = G0.forward(v)
        x_ref = torch.zeros(G0.vol_shape, device="cuda")
        st = tigre.tigre_cgls_begin(G0.handle, b, x_ref, x0_zero=True)
        tigre.tigre_cgls_iterate(st, 4)
        h_ref = tigre.tigre_cgls_history(st, 4)
        tigre.tigre_cgls_end(st)
    s = torch.cuda.Stream()
    torch.cuda.synchronize()
    with torch.cuda.stream(s), tigre.Geometry(geo, ang) as G:
        tigre.tigre_geometry_set_brick(G.handle, 16)
        x = torch.zeros(G.vol_shape, device="cuda")
        st = tigre.tigre_cgls_begin(G.handle, b, x, stream=s, graph=True, x0_zero=True)
        tigre.tigre_cgls_iterate(st, 4)
        h = tigre.tigre_cgls_history(st, 4)
        tigre.tigre_cgls_end(st)
        torch.cuda.synchronize()
    assert torch.equal(x, x_ref)
    np.testing.assert_array_equal(h, h_ref)


def test_graph_replay_after_the_handle_served_another_storage_type(tigre):
    """Between replays, a call on the same handle in BF16 re-lays the cached
    forward workspaces out for 16-bit elements.  The next replay restores
    the F32 layout (and recaptures if an address changed): the run equals
    an uninterrupted eager run bit for bit."""
    geo, ang, vol = case()
    v = torch.from_numpy(vol).cuda()
    with tigre.Geometry(geo, ang) as G0:
        b = G0.forward(v)
        x_ref = torch.zeros(G0.vol_shape, device="cuda")
        st = tigre.tigre_cgls_begin(G0.handle, b, x_ref)
        tigre.tigre_cgls_iterate(st, 4)
        h_ref = tigre.tigre_cgls_history(st, 4)
        tigre.tigre_cgls_end(st)
    s = torch.cuda.Stream()
    torch.cuda.synchronize()
    with torch.cuda.stream(s), tigre.Geometry(geo, ang) as G:
        x = torch.zeros(G.vol_shape, device="cuda")
        st = tigre.tigre_cgls_begin(G.handle, b, x, stream=s, graph=True)
        tigre.tigre_cgls_iterate(st, 2)
        G.forward(v.bfloat16())  # same handle, other storage type, same stream
        G.backward(b.half())
        tigre.tigre_cgls_iterate(st, 2)
        h = tigre.tigre_cgls_history(st, 4)
        tigre.tigre_cgls_end(st)
        torch.cuda.synchronize()
    assert torch.equal(x, x_ref)
    np.testing.assert_array_equal(h, h_ref)


def test_resume_rejects_a_search_direction_buffer_smaller_than_p(tigre):
    """The C entry point itself refuses a p buffer below the volume's bytes
    (with a large enough r) before copying anything."""
    import ctypes
    geo, ang, _ = case()
    with tigre.Geometry(geo, ang) as G:
        b = torch.zeros(G.proj_shape, device="cuda")
        x = torch.zeros(G.vol_shape, device="cuda")
        r = torch.zeros(G.proj_shape)
        p = torch.zeros(G.vol_shape)
        o = tigre._opts(8, None)
        out = ctypes.c_void_p()
        st = tigre._lib.tigre_cgls_resume(
            G.handle, ctypes.c_void_p(b.data_ptr()), ctypes.c_void_p(x.data_ptr()),
            ctypes.c_void_p(r.data_ptr()), r.numel() * 4, ctypes.c_void_p(p.data_ptr()), 4,
            1.0, ctypes.byref(o), ctypes.byref(out))
        assert st == tigre.TIGRE_ERR_INVALID_ARG
        assert out.value is None
        assert b"smaller" in tigre._lib.tigre_last_error()


def test_resume_rejects_bad_checkpoints(tigre):
    geo, ang, _ = case()
    with tigre.Geometry(geo, ang) as G:
        b = torch.zeros(G.proj_shape, device="cuda")
        x = torch.zeros(G.vol_shape, device="cuda")
        r = torch.zeros(G.proj_shape)
        p = torch.zeros(G.vol_shape)
        with pytest.raises(tigre.TigreError):
            tigre.tigre_cgls_resume(G.handle, b, x, r, p, float("nan"))
        with pytest.raises(TypeError):
            tigre.tigre_cgls_resume(G.handle, b, x, r.bfloat16(), p, 1.0)
        with pytest.raises(ValueError):
            tigre.tigre_cgls_resume(G.handle, b, x, r[:1], p, 1.0)


@pytest.mark.parametrize("host", [False, True])
def test_x0_zero_flag_gives_the_zero_start_bits(tigre, host):
    """TIGRE_X0_ZERO: vol is not read (here it holds garbage), q = 0 replaces
    the projection of x0; the iterates and residuals are the bits of a run
    from an explicit zero x0."""
    geo, ang, vol = case()
    with tigre.Geometry(geo, ang) as G:
        b = G.forward(torch.from_numpy(vol).cuda())
        dev = "cpu" if host else "cuda"
        bb = b.cpu() if host else b
        x_ref = torch.zeros(G.vol_shape, device=dev)
        h_ref = tigre.tigre_cgls(G.handle, bb, x_ref, 5, host=host)
        x = torch.full(G.vol_shape, float("nan"), device=dev)
        h = tigre.tigre_cgls(G.handle, bb, x, 5, host=host, x0_zero=True)
        torch.cuda.synchronize()
    np.testing.assert_array_equal(h, h_ref)
    assert torch.equal(x.cpu(), x_ref.cpu())


def test_x0_zero_stepwise_and_refusals(tigre):
    geo, ang, vol = case()
    with tigre.Geometry(geo, ang) as G:
        b = G.forward(torch.from_numpy(vol).cuda())
        x_ref = torch.zeros(G.vol_shape, device="cuda")
        st = tigre.tigre_cgls_begin(G.handle, b, x_ref)
        tigre.tigre_cgls_iterate(st, 3)
        h_ref = tigre.tigre_cgls_history(st, 3)
        tigre.tigre_cgls_end(st)
        x = torch.full(G.vol_shape, 7.0, device="cuda")
        st = tigre.tigre_cgls_begin(G.handle, b, x, x0_zero=True)
        tigre.tigre_cgls_iterate(st, 3)
        h = tigre.tigre_cgls_history(st, 3)
        tigre.tigre_cgls_end(st)
        torch.cuda.synchronize()
        assert torch.equal(x, x_ref)
        np.testing.assert_array_equal(h, h_ref)
        with pytest.raises(tigre.TigreError):  # out of core reads x0 from the host volume
            tigre.tigre_cgls(G.handle, b.cpu(), torch.zeros(G.vol_shape), 1, out_of_core=True,
                             x0_zero=True)



def test_save_rejects_buffers_smaller_than_the_state(tigre):
    geo, ang, _ = case()
    with tigre.Geometry(geo, ang) as G:
        b = torch.zeros(G.proj_shape, device="cuda")
        x = torch.zeros(G.vol_shape, device="cuda")
        st = tigre.tigre_cgls_begin(G.handle, b, x)
        try:
            with pytest.raises(tigre.TigreError):
                tigre.tigre_cgls_save(st, torch.empty(10), torch.empty(G.vol_shape))
            with pytest.raises(tigre.TigreError):  # half the bytes of the F32 state's p
                tigre.tigre_cgls_save(st, torch.empty(G.proj_shape),
                                      torch.empty(G.vol_shape, dtype=torch.bfloat16))
        finally:
            tigre.tigre_cgls_end(st)
