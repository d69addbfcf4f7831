"""The continuous-batching server: every request's result in the mix (packed with
others into shared launches, overlapping on the device) is bit-identical to the
request solved alone, and the server honours its memory budget."""
import numpy as np
import pytest
import torch

from paper_2609_02876_gb300 import api, build, serve

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def _alone(r):
    t0, t1, save_t, atol_fixed, ratio = serve._spec(r.problem)
    atol = r.rtol * ratio if ratio is not None else atol_fixed
    P = torch.as_tensor(np.ascontiguousarray(r.params.T), device="cuda")
    Y = torch.as_tensor(np.ascontiguousarray(r.y0.T), device="cuda")
    res = api.solve_grad(r.problem, P, Y, t0, t1, save_t, r.rtol, atol, layout="soa", check=False)
    return {k: v.cpu().numpy() for k, v in res.items() if k in ("loss", "params_bar", "y0_bar", "status")}


def test_results_in_the_mix_equal_results_alone():
    reqs = serve.c4_stream(30, seed=3, log2n=(5, 12))
    server = serve.Server(slots=3, budget_bytes=1 << 30, max_pack=1 << 13)
    try:
        serve.run_stream(server, reqs, rate=None)
    finally:
        server.close()
    packed = [b for b in server.batch_log if b[2] > 1]
    assert packed, "expected some launches to pack several requests"
    for r in reqs:
        a = _alone(r)
        assert (r.status == 0).all()
        np.testing.assert_array_equal(r.status, a["status"])
        np.testing.assert_array_equal(r.loss, a["loss"])
        np.testing.assert_array_equal(r.params_bar, a["params_bar"].T)
        np.testing.assert_array_equal(r.y0_bar, a["y0_bar"].T)


def test_budget_admits_one_batch_at_a_time_when_tight():
    reqs = serve.c4_stream(8, seed=5, log2n=(8, 10))
    server = serve.Server(slots=4, budget_bytes=1, max_pack=1 << 10)
    try:
        serve.run_stream(server, reqs, rate=None)
    finally:
        server.close()
    spans = sorted((b[4], b[5]) for b in server.batch_log)
    for (s0, e0), (s1, e1) in zip(spans, spans[1:]):
        assert s1 >= e0 - 1e-3, "batches overlapped although the budget admits one at a time"
    assert all((r.status == 0).all() for r in reqs)


def test_chunked_large_requests_equal_results_alone():
    """Requests larger than max_chunk run as several launches (chunks), small ones
    pass them at chunk boundaries; every request's results still equal its own
    solve alone bit for bit."""
    reqs = serve.c4_stream(12, seed=9, log2n=(6, 12))
    server = serve.Server(slots=3, budget_bytes=1 << 30, max_pack=1 << 13, max_chunk=700)
    try:
        serve.run_stream(server, reqs, rate=None)
    finally:
        server.close()
    assert any(r.n > 700 for r in reqs)
    assert len(server.batch_log) > len([r for r in reqs if r.n <= 700])
    for r in reqs:
        a = _alone(r)
        assert (r.status == 0).all()
        np.testing.assert_array_equal(r.loss, a["loss"])
        np.testing.assert_array_equal(r.params_bar, a["params_bar"].T)
        np.testing.assert_array_equal(r.y0_bar, a["y0_bar"].T)
