"""Host logic of the forward projector's angle groups (no GPU): the table
the angle-paired warps read holds every angle exactly once, each group in
one memory layout and one march direction with neighbouring angles, and the
automatic path pairs angles only while the rays of one pixel at paired
angles stay within 16 voxels of each other."""
import numpy as np
import pytest

from paper_1905_03748_gb300 import synth


@pytest.fixture(scope="module")
def tigre():
    from paper_1905_03748_gb300 import tigre as t
    return t


def angle_class(t):
    """(layout, march direction): layout 1 when |cos| > |sin| (rays of a
    detector row spread along y), direction = sign of the source along the
    layout's depth axis."""
    layout = int(abs(np.cos(t)) > abs(np.sin(t)))
    main = np.cos(t) if layout else np.sin(t)
    return layout, bool(main > 0)


def check_table(tab, ang):
    flat = tab[tab >= 0]
    assert sorted(flat.tolist()) == list(range(len(ang)))  # every angle exactly once
    for grp in tab:
        assert grp[0] >= 0                                  # a group's first slot holds an angle
        idx = grp[grp >= 0]
        assert (grp[len(idx):] == -1).all()                 # padding only at the end
        assert len({angle_class(ang[i]) for i in idx}) == 1


@pytest.mark.parametrize("name,na,drift,pairs", [("cgls_512", 360, 6.32, True),
                                                 ("mixed_1024", 720, 6.32, True),
                                                 ("mixed_1024", 360, 12.64, True),
                                                 ("mixed_1024", 90, 50.56, False)])
def test_uniform_angles(tigre, name, na, drift, pairs):
    geo, _ = synth.workload(name)
    ang = synth.angles(na)
    for size in (2, 4):
        tab, d, auto = tigre.tigre_forward_angle_groups(geo, ang, size)
        check_table(tab, ang)
        assert d == pytest.approx(drift, rel=2e-3)
        assert auto == pairs
        # neighbours: inside a full group the angles are consecutive steps
        step = 2 * np.pi / na
        for grp in tab:
            if (grp >= 0).all():
                gaps = np.abs(np.remainder(np.diff(ang[grp]) + np.pi, 2 * np.pi) - np.pi)
                np.testing.assert_allclose(gaps, step, rtol=1e-9)


def test_any_angle_set(tigre):
    geo = synth.geometry((37, 29, 21), (1.0, 0.9, 1.1), (53, 27), (1.05, 0.95), dso=300.0,
                         dsd=450.0, off_origin=(0.5, -0.3, 0.2))
    rng = np.random.default_rng(12)
    ang = rng.uniform(-3 * np.pi, 3 * np.pi, 29)
    ang = np.concatenate([ang, ang[3:4]])
    for size in (2, 4):
        tab, d, _ = tigre.tigre_forward_angle_groups(geo, ang, size)
        check_table(tab, ang)
        assert np.isfinite(d) and d >= 0


def test_one_angle_and_refusals(tigre):
    geo, _ = synth.workload("small_64")
    tab, d, auto = tigre.tigre_forward_angle_groups(geo, [0.3], 2)
    assert tab.tolist() == [[0, -1]] and d == 0.0 and not auto
    for bad in ([float("nan")], []):
        with pytest.raises(tigre.TigreError):
            tigre.tigre_forward_angle_groups(geo, bad, 2)
    with pytest.raises(tigre.TigreError):
        tigre.tigre_forward_angle_groups(geo, [0.1, 0.2], 3)
