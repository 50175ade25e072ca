"""Autograd through the projector: dot-product test, finite differences,
gradient against the FP64 oracle, and the 512^3 x 360 dot test."""
import numpy as np
import pytest
import torch

import oracle
from paper_1905_03748_gb300 import synth

pytestmark = pytest.mark.gpu


def small_geo():
    geo = synth.geometry((20, 18, 14), (1.0, 1.1, 0.9), (31, 21), (1.0, 1.0), dso=150.0,
                         dsd=240.0, off_origin=(0.3, 0.0, -0.2), off_det=(0.4, 0.1))
    return geo, np.sort(np.random.default_rng(1).uniform(0, 2 * np.pi, 9))


def test_gradient_equals_oracle_adjoint_of_residual(tigre):
    from paper_1905_03748_gb300.autograd import forward_project
    geo, ang = small_geo()
    x_np = synth.random_volume((14, 18, 20), seed=2)
    b_np = np.random.default_rng(3).random((9, 21, 31)).astype(np.float32)
    with tigre.Geometry(geo, ang) as G:
        x = torch.from_numpy(x_np).cuda().requires_grad_(True)
        b = torch.from_numpy(b_np).cuda()
        loss = 0.5 * ((forward_project(x, G) - b) ** 2).sum()
        loss.backward()
        grad = x.grad.double().cpu().numpy()
    ref = oracle.adjoint(geo, ang, oracle.forward(geo, ang, x_np) - b_np)
    assert np.linalg.norm(grad - ref) / np.linalg.norm(ref) < 1e-4


def test_central_finite_differences(tigre):
    """L(x) = 0.5 ||A x - b||^2 is quadratic, so the central difference along
    any direction equals <grad, v> up to rounding."""
    from paper_1905_03748_gb300.autograd import forward_project
    geo, ang = small_geo()
    rng = np.random.default_rng(4)
    with tigre.Geometry(geo, ang) as G:
        x = torch.from_numpy(synth.random_volume((14, 18, 20), seed=5)).cuda()
        b = torch.from_numpy(rng.random((9, 21, 31)).astype(np.float32)).cuda()
        xr = x.clone().requires_grad_(True)
        L = lambda z: 0.5 * ((forward_project(z, G).double() - b.double()) ** 2).sum()  # noqa
        L(xr).backward()
        for seed in range(3):
            v = torch.from_numpy(np.random.default_rng(10 + seed).standard_normal(x.shape)
                                 .astype(np.float32)).cuda()
            eps = 1e-2
            fd = (L(x + eps * v) - L(x - eps * v)) / (2 * eps)
            an = (xr.grad.double() * v.double()).sum()
            assert abs(float(fd) - float(an)) / abs(float(an)) < 1e-4


def test_adjoint_function_backward_is_forward(tigre):
    from paper_1905_03748_gb300.autograd import adjoint_project, forward_project
    geo, ang = small_geo()
    with tigre.Geometry(geo, ang) as G:
        y = torch.from_numpy(np.random.default_rng(6).random((9, 21, 31)).astype(np.float32)).cuda()
        x = torch.from_numpy(synth.random_volume((14, 18, 20), seed=7)).cuda()
        yr = y.clone().requires_grad_(True)
        (adjoint_project(yr, G) * x).sum().backward()
        assert torch.allclose(yr.grad, forward_project(x, G), rtol=1e-6, atol=1e-6)


def test_dot_product_at_full_workload(tigre):
    """<A x, y> = <x, A^T y> on the 512^3 x 360 workload through autograd."""
    from paper_1905_03748_gb300.autograd import forward_project
    geo, ang = synth.workload("cgls_512")
    with tigre.Geometry(geo, ang) as G:
        gen = torch.Generator(device="cuda").manual_seed(0)
        x = torch.rand(G.vol_shape, device="cuda", generator=gen).requires_grad_(True)
        y = torch.rand(G.proj_shape, device="cuda", generator=gen)
        lhs = (forward_project(x, G).double() * y.double()).sum()
        lhs.backward(retain_graph=False)
        # d<Ax, y>/dx = A^T y
        rhs = (x.detach().double() * x.grad.double()).sum()
        assert abs(float(lhs.detach()) - float(rhs)) / abs(float(lhs.detach())) < 1e-5
