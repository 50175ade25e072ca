"""Host logic of the continuous-batching server (no GPU): HBM footprints,
the admission policy (slots, HBM budget, arrival order or least work first),
seeded Poisson arrivals and the latency summary."""
import numpy as np
import pytest
import torch

from paper_1905_03748_gb300 import synth


@pytest.fixture(scope="module")
def serving():
    from paper_1905_03748_gb300 import serving as s
    return s


def request(serving, rid, n, na=30, dtype=torch.float32, arrival=0.0, n_iter=15):
    geo = synth.cube_geometry(n, n, fov_mm=64.0)
    proj = torch.zeros((na, n, n), dtype=dtype)
    return serving.Request(rid, geo, synth.angles(na), proj, n_iter, arrival)


def test_footprint_counts_six_vectors_layouts_and_slack(serving):
    geo, ang = synth.workload("small_64")
    # x, p, s: 3 x 64^3 and b, r, q: 3 x 100 x 128^2 values of the storage
    # type; 16-byte quads: the backprojector's 100 x (128 + 4) x (128 + 12 + 8)
    # and the two zero-bordered layouts' 2 x 68^3; 64 MiB slack
    vectors = 3 * 64 ** 3 + 3 * 100 * 128 ** 2
    quads = 16 * (100 * 132 * 148 + 2 * 68 ** 3)
    assert serving.footprint_bytes(geo, len(ang)) == 4 * vectors + quads + (64 << 20)
    assert serving.footprint_bytes(geo, len(ang), 2) == 2 * vectors + quads + (64 << 20)


def test_storage_type_follows_the_projections(serving):
    assert serving.storage_dtype(request(serving, 0, 16, dtype=torch.bfloat16)) == torch.bfloat16
    assert serving.storage_dtype(request(serving, 0, 16, dtype=torch.float64)) == torch.float32
    small = serving.request_bytes(request(serving, 0, 32, dtype=torch.float16))
    assert small < serving.request_bytes(request(serving, 0, 32))


def test_fifo_admits_in_order_within_slots_and_budget(serving):
    reqs = [request(serving, i, n) for i, n in enumerate([32, 32, 48, 16])]
    sizes = [serving.request_bytes(r) for r in reqs]
    # budget for the first two only: the 48^3 request at the head blocks the 16^3 one
    q = list(reqs)
    got = serving.admit(q, 0, 0, 8, sizes[0] + sizes[1] + sizes[2] // 2)
    assert [r.rid for r in got] == [0, 1] and [r.rid for r in q] == [2, 3]
    # slots bound admission too
    q = list(reqs)
    got = serving.admit(q, 6, 0, 8, 10 ** 12)
    assert [r.rid for r in got] == [0, 1]
    # memory already in use counts
    q = list(reqs)
    assert serving.admit(q, 1, 10 ** 12, 8, 10 ** 12) == [] and len(q) == 4


def test_a_request_larger_than_the_budget_runs_alone(serving):
    big = request(serving, 0, 64)
    q = [big, request(serving, 1, 16)]
    got = serving.admit(q, 0, 0, 8, 1000)
    assert [r.rid for r in got] == [0]          # nothing resident: admitted alone
    q = [request(serving, 2, 64)]
    assert serving.admit(q, 1, 0, 8, 1000) == []  # waits while anything is resident


def test_sjf_admits_least_work_first(serving):
    reqs = [request(serving, 0, 48, arrival=0.0), request(serving, 1, 16, arrival=0.1),
            request(serving, 2, 32, arrival=0.2), request(serving, 3, 16, na=18, arrival=0.3)]
    q = list(reqs)
    got = serving.admit(q, 0, 0, 2, 10 ** 12, policy="sjf")
    assert [r.rid for r in got] == [3, 1] and [r.rid for r in q] == [2, 0]
    with pytest.raises(ValueError):
        serving.Server.__init__(object.__new__(serving.Server), policy="lifo")


def test_poisson_arrivals_are_seeded_and_increasing(serving):
    def make(i, rng):
        geo = synth.cube_geometry(16, 16)
        return geo, synth.angles(8), torch.zeros((8, 16, 16)), 3

    a = serving.poisson_requests(200, 20.0, 5, make)
    b = serving.poisson_requests(200, 20.0, 5, make)
    t = np.array([r.arrival for r in a])
    assert np.array_equal(t, [r.arrival for r in b])
    assert (np.diff(t) > 0).all() and t[0] > 0
    assert 0.035 < np.diff(t).mean() < 0.065  # mean gap 1 / rate


def test_latency_summary(serving):
    res = [serving.Result(i, None, None, arrival=float(i), admitted=float(i),
                          finished=float(i) + 1.0 + (i == 9) * 9.0) for i in range(10)]
    st = serving.latency_stats(res)
    assert st["p50_s"] == pytest.approx(1.0)
    assert st["p99_s"] > 9.0 and st["mean_s"] == pytest.approx(1.9)
    assert st["makespan_s"] == pytest.approx(19.0)
    assert st["throughput_req_s"] == pytest.approx(10 / 19.0)


def test_batch_key_separates_what_cannot_share_a_batch(serving):
    a = request(serving, 0, 16)
    assert serving.batch_key(a) == serving.batch_key(request(serving, 1, 16, arrival=3.0))
    assert serving.batch_key(a) != serving.batch_key(request(serving, 2, 24))
    assert serving.batch_key(a) != serving.batch_key(request(serving, 3, 16, na=31))
    assert serving.batch_key(a) != serving.batch_key(request(serving, 4, 16, dtype=torch.bfloat16))
    assert serving.batch_key(a) != serving.batch_key(request(serving, 5, 16, n_iter=14))


def test_groups_take_same_key_requests_from_behind_the_head(serving):
    sizes = [16, 24, 16, 16, 24, 16, 16]
    reqs = [request(serving, i, n) for i, n in enumerate(sizes)]
    q = list(reqs)
    got = serving.admit_groups(q, 0, 0, 8, 10 ** 12, "fifo", 3)
    # head 0 takes 2 and 3 (max 3 per group); head 1 takes 4; head 5 takes 6
    assert [[r.rid for r in g] for g in got] == [[0, 2, 3], [1, 4], [5, 6]] and q == []
    # slots count requests: 4 slots stop inside the second group
    q = list(reqs)
    got = serving.admit_groups(q, 0, 0, 4, 10 ** 12, "fifo", 3)
    assert [[r.rid for r in g] for g in got] == [[0, 2, 3], [1]]
    assert [r.rid for r in q] == [4, 5, 6]
    # one member per group is plain admission
    q = list(reqs)
    assert [[r.rid for r in g] for g in serving.admit_groups(q, 0, 0, 2, 10 ** 12)] == [[0], [1]]
    # the budget stops followers too
    q = list(reqs)
    one = serving.request_bytes(reqs[0])
    got = serving.admit_groups(q, 0, 0, 8, 2 * one, "fifo", 4)
    assert [[r.rid for r in g] for g in got] == [[0, 2]]
