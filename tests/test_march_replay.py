"""The CPU replay of the forward projector's march (host only): with two
neighbouring angles per warp, interleaving them over the lanes (each 16-lane
half holds 8 pixels of both) touches fewer 128-byte lines per half-warp than
16 pixels of one angle per half, while the whole-warp line count and the
lanes taking a sample are the same for both orders."""
import sys
from pathlib import Path

import numpy as np

sys.path.insert(0, str(Path(__file__).resolve().parents[1]))
from paper_1905_03748_gb300 import march_replay, synth  # noqa: E402


def test_interleaved_pairs_touch_fewer_lines_per_half_warp():
    geo, ang = synth.workload("cgls_512")
    blocked = march_replay.replay(geo, ang, 2, "blocked", n_warps=30, seed=3)
    inter = march_replay.replay(geo, ang, 2, "interleaved", n_warps=30, seed=3)
    assert blocked["requests"] == inter["requests"] > 0
    assert np.isclose(blocked["lines_per_request"], inter["lines_per_request"])
    assert np.isclose(blocked["lanes_per_request"], inter["lanes_per_request"])
    assert inter["halfwarp_lines_per_request"] < 0.9 * blocked["halfwarp_lines_per_request"]
    # two halves, each touching at least one line
    assert inter["halfwarp_lines_per_request"] >= 2.0


def test_rays_take_the_sample_count_of_the_midpoint_rule():
    """A ray through the centre of a 64^3 cube along x: its clip to the
    support [-1, 64] is 65 voxels, i.e. 130 samples of half a voxel."""
    geo = synth.geometry(64, 1.0, (65, 65), 1.0, dso=1000.0, dsd=1500.0)
    x0, dx, K, lay = march_replay.rays(geo, 0.0, np.array([32.0]), 32)
    assert lay == 1 and K[0] == 130
    assert np.isclose(abs(dx[0, 1]), 0.5) and np.allclose(dx[0, [0, 2]], 0.0)
