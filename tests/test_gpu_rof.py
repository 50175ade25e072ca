"""GPU parity of the ROF-model TV minimiser against the FP64 oracle."""
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


@pytest.mark.parametrize("shape", [(21, 29, 37), (1, 17, 40), (33, 8, 1)])
def test_rof_matches_oracle(tigre, shape):
    """Ragged sizes, including one-voxel axes (no differences along them)."""
    f = synth.random_volume(shape, seed=16)
    ref = oracle.rof_denoise(f, 3.0, 40)
    got = tigre.tigre_rof_denoise(torch.from_numpy(f).cuda(), 3.0, 40).cpu().numpy()
    assert rel(got, ref) < 1e-5


def test_rof_in_place_and_zero_iterations(tigre):
    f = synth.random_volume((9, 10, 11), seed=17)
    t = torch.from_numpy(f.copy()).cuda()
    ref = oracle.rof_denoise(f, 2.0, 25)
    tigre.tigre_rof_denoise(t, 2.0, 25, out=t)
    assert rel(t.cpu().numpy(), ref) < 1e-5
    z = tigre.tigre_rof_denoise(torch.from_numpy(f).cuda(), 2.0, 0).cpu().numpy()
    np.testing.assert_array_equal(z, f)


def test_rof_solves_the_two_level_step(tigre):
    f = np.zeros((2, 3, 16), np.float32)
    f[:, :, 6:] = 1.0
    u = tigre.tigre_rof_denoise(torch.from_numpy(f).cuda(), 1.0, 1500).cpu().numpy()
    np.testing.assert_allclose(u[:, :, :6], 1.0 / 6, atol=1e-5)
    np.testing.assert_allclose(u[:, :, 6:], 0.9, atol=1e-5)


def test_rof_rejects_bad_arguments(tigre):
    f = torch.zeros((4, 4, 4), device="cuda")
    with pytest.raises(tigre.TigreError):
        tigre.tigre_rof_denoise(f, 0.0, 3)
    with pytest.raises(tigre.TigreError):
        tigre.tigre_rof_denoise(f, 1.0, -1)
