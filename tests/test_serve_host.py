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
    return serve.pack_batch(collections.deque(serve.Item(r, 0, r.n) for r in queue), max_pack)


def test_packing_takes_the_oldest_key_in_arrival_order_up_to_the_limit():
    q = [req(0, "lorenz", 100, 1e-6), req(1, "vdp", 50, 1e-6), req(2, "lorenz", 300, 1e-6),
         req(3, "lorenz", 100, 1e-8), req(4, "lorenz", 700, 1e-6), req(5, "lorenz", 50, 1e-6)]
    batch, total = take(q, 1000)
    assert [it.req.rid for it in batch] == [0, 2, 5]  # 4 would pass the limit; 1 and 3 have other keys
    assert total == 450
    batch, total = take(q, 10 ** 6)
    assert [it.req.rid for it in batch] == [0, 2, 4, 5] and total == 1150


def test_an_oversized_request_still_runs_alone():
    batch, total = take([req(7, "hires", 5000, 1e-6), req(8, "hires", 10, 1e-6)], 1000)
    assert [it.req.rid for it in batch] == [7] and total == 5000


def test_large_requests_are_chunked_and_small_ones_pass_them():
    """Submitting splits a request beyond max_chunk into chunks queued in arrival
    order; the scheduler's pick serves queued small requests first and then the
    oldest chunk."""
    fake = types.SimpleNamespace(max_chunk=1000, max_pack=1000, _small=collections.deque(),
                                 _large=collections.deque(), _closed=False,
                                 _cv=__import__("threading").Condition())
    big, small, big2 = req(0, "lorenz", 2500, 1e-6), req(1, "vdp", 10, 1e-6), req(2, "lorenz", 1200, 1e-6)
    for r in (big, small, big2):
        serve.Server.submit(fake, r)
    assert big.left == 3 and small.left == 1 and big2.left == 2
    assert [(it.req.rid, it.lo, it.hi) for it in fake._large] == [(0, 0, 1000), (0, 1000, 2000), (0, 2000, 2500),
                                                                  (2, 0, 1000), (2, 1000, 1200)]
    (batch, total), q = serve.Server._take_batch(fake)
    assert q is fake._small and [it.req.rid for it in batch] == [1] and total == 10
    fake._small.clear()
    (batch, total), q = serve.Server._take_batch(fake)
    assert q is fake._large and [(it.req.rid, it.lo) for it in batch] == [(0, 0)] and total == 1000
    assert big.params_bar.shape == (2500, 1) and big.y0_bar.shape == (2500, 2)  # results filled by slices


def test_serving_stream_follows_its_distribution():
    reqs = serve.c4_stream(200, seed=3, log2n=(6, 12))
    sizes = np.array([r.n for r in reqs])
    assert sizes.min() >= 64 and sizes.max() <= 4096
    assert {r.problem for r in reqs} == {"lorenz", "vdp", "robertson"}
    assert {r.rtol for r in reqs} == {1e-6, 1e-8}
    assert [r.rid for r in reqs] == list(range(200))
    again = serve.c4_stream(200, seed=3, log2n=(6, 12))
    assert all(np.array_equal(a.params, b.params) for a, b in zip(reqs, again))  # seeded
