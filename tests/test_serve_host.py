"""Host-side logic of the request server, on the CPU: the record-footprint
estimate used for admission, the packing rule (oldest request first, same
(problem, rtol) behind it, up to the pack limit, FIFO within a key) and the
shape of the serving stream."""
import collections
import types

import numpy as np
import pytest

from paper_2609_02876_gb300 import build
from paper_2609_02876_gb300 import serve


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()  # problem_info comes from the C-ABI library (no GPU call)


def req(rid, problem, n, rtol):
    return serve.Request(rid, problem, np.zeros((n, 1)), np.zeros((n, 2)), rtol)


def test_record_footprint_scales_with_size_and_tolerance():
    a = serve.record_footprint("lorenz", 1000, 1e-6)
    assert serve.record_footprint("lorenz", 2000, 1e-6) > 1.99 * a
    # the order-5 step-count law: 100x tighter rtol -> 100^(1/5) = 2.5x the steps
    ratio = serve.record_footprint("lorenz", 1000, 1e-8) / a
    assert 2.3 < ratio < 2.6
    assert serve.record_footprint("robertson", 1000, 1e-6) > a  # more steps per trajectory


def take(queue, max_pack):
    fake = types.SimpleNamespace(_queue=collections.deque(queue), max_pack=max_pack)
    return serve.Server._take_batch(fake)


def test_packing_takes_the_oldest_key_in_arrival_order_up_to_the_limit():
    q = [req(0, "lorenz", 100, 1e-6), req(1, "vdp", 50, 1e-6), req(2, "lorenz", 300, 1e-6),
         req(3, "lorenz", 100, 1e-8), req(4, "lorenz", 700, 1e-6), req(5, "lorenz", 50, 1e-6)]
    batch, total = take(q, 1000)
    assert [r.rid for r in batch] == [0, 2, 5]  # 4 would pass the limit; 1 and 3 have other keys
    assert total == 450
    batch, total = take(q, 10 ** 6)
    assert [r.rid for r in batch] == [0, 2, 4, 5] and total == 1150


def test_an_oversized_request_still_runs_alone():
    batch, total = take([req(7, "hires", 5000, 1e-6), req(8, "hires", 10, 1e-6)], 1000)
    assert [r.rid for r in batch] == [7] and total == 5000


def test_serving_stream_follows_its_distribution():
    reqs = serve.c4_stream(200, seed=3, log2n=(6, 12))
    sizes = np.array([r.n for r in reqs])
    assert sizes.min() >= 64 and sizes.max() <= 4096
    assert {r.problem for r in reqs} == {"lorenz", "vdp", "robertson"}
    assert {r.rtol for r in reqs} == {1e-6, 1e-8}
    assert [r.rid for r in reqs] == list(range(200))
    again = serve.c4_stream(200, seed=3, log2n=(6, 12))
    assert all(np.array_equal(a.params, b.params) for a, b in zip(reqs, again))  # seeded
