"""GPU parity of the Robertson neural right-hand side (shared-weight MLP in a
stiff system) against the FP64 oracle on the GPU's own recorded mesh, for
Rodas5P and Rosenbrock23.

Per-trajectory results are FP64 on both sides. States and losses: normwise
relative error per trajectory vector 1e-10 (the GPU's tanh, exp and log1p are
the CUDA library's, the oracle's the C library's; both within an ulp or two,
and the stiff replay carries those differences). Gradients: the problem's own
rounding floor is measured first, as the normwise disagreement of two exact
FP64 evaluations of the same derivative in the oracle (forward-mode JVP along
each input against the adjoint, on the same mesh); it reaches 1.8e-10 for
Rodas5P here, so the bound is max(1e-10, 20 x floor). The shared-weight
gradient is an FP64 sum on the GPU written out in FP32: normwise 1e-6.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2609_02876_gb300 import api, build
from paper_2609_02876_gb300 import workloads as W
from tests.test_gpu_tsit5 import assert_close, dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def rounding_floor(wl, off, h, om):
    """Normwise fwd-vs-rev disagreement of the oracle's gradient: (theta_bar floor, y0_bar floor),
    each relative to the max norm of its own vector, as the comparisons below are."""
    g = oracle.replay_grad("nrob", wl["params"], wl["y0"], wl["t0"], wl["t1"], wl["save_t"], off, h, method=om,
                           w=wl["w"])
    n, P = wl["params"].shape
    d = wl["y0"].shape[1]
    floors = []
    for vec, width, on_theta in ((g["params_bar"], P, True), (g["y0_bar"], d, False)):
        worst = np.zeros(n)
        for q in range(width):
            pd, yd = np.zeros((n, P)), np.zeros((n, d))
            (pd if on_theta else yd)[:, q] = 1.0
            j = oracle.replay_jvp("nrob", wl["params"], wl["y0"], wl["t0"], wl["t1"], wl["save_t"], off, h, pd, yd,
                                  method=om, w=wl["w"])
            worst = np.maximum(worst, np.abs(j["loss_dot"] - vec[:, q]) / np.abs(vec).max(1))
        floors.append(worst.max())
    return floors


def workload(n):
    wl = W.make("nrob", n)
    w32 = np.asarray(wl["w"], dtype=np.float32)
    return dict(wl, w=w32.astype(np.float64)), torch.as_tensor(w32, device="cuda")


@pytest.mark.parametrize("method,om", [("rodas5p", oracle.METHOD_RODAS5P),
                                       ("rosenbrock23", oracle.METHOD_ROSENBROCK23)])
def test_nrob_record_and_reverse_match_oracle(method, om):
    n = 96
    wl, SW = workload(n)
    P, Y = dev(wl["params"].T), dev(wl["y0"].T)
    rec, ysv, st = api.forward_record("nrob", P, Y, wl["t0"], wl["t1"], wl["save_t"], wl["rtol"], wl["atol"],
                                      layout="soa", shared_w=SW, method=method)
    assert (st.cpu().numpy() == 0).all()
    np.testing.assert_allclose(ysv.cpu().numpy().sum(1), 1.0, atol=1e-12)  # mass
    g = api.reverse(rec, P, Y, layout="soa", shared_w=SW)
    off, h = rec.export_mesh()
    o = oracle.replay_grad("nrob", wl["params"], wl["y0"], wl["t0"], wl["t1"], wl["save_t"], off, h, method=om,
                           w=wl["w"])
    assert o["ok"].all()
    assert_close(ysv.permute(2, 0, 1).cpu().numpy(), o["y_save"], "y_save", rtol=1e-10)
    assert_close(g["loss"].cpu().numpy(), o["loss"], "loss", rtol=1e-10)
    fp, fy = rounding_floor(wl, off, h, om)
    assert_close(g["params_bar"].cpu().numpy().T, o["params_bar"], "params_bar", rtol=max(1e-10, 20.0 * fp))
    assert_close(g["y0_bar"].cpu().numpy().T, o["y0_bar"], "y0_bar", rtol=max(1e-10, 20.0 * fy))
    wb = g["shared_w_bar"].cpu().numpy().astype(np.float64)
    err = np.abs(wb - o["w_bar"]).max() / np.abs(o["w_bar"]).max()
    assert err <= 1e-6, err


def test_nrob_weight_gradient_is_deterministic_and_solve_grad_agrees():
    n = 200
    wl, SW = workload(n)
    P, Y = dev(wl["params"].T), dev(wl["y0"].T)
    a = api.solve_grad("nrob", P, Y, wl["t0"], wl["t1"], wl["save_t"], wl["rtol"], wl["atol"], layout="soa",
                       shared_w=SW, method="rosenbrock23")
    b = api.solve_grad("nrob", P, Y, wl["t0"], wl["t1"], wl["save_t"], wl["rtol"], wl["atol"], layout="soa",
                       shared_w=SW, method="rosenbrock23")
    np.testing.assert_array_equal(a["shared_w_bar"].cpu().numpy(), b["shared_w_bar"].cpu().numpy())
    np.testing.assert_array_equal(a["params_bar"].cpu().numpy(), b["params_bar"].cpu().numpy())
    rec, _, _ = api.forward_record("nrob", P, Y, wl["t0"], wl["t1"], wl["save_t"], wl["rtol"], wl["atol"],
                                   layout="soa", shared_w=SW, method="rosenbrock23", want_saves=False)
    g = api.reverse(rec, P, Y, layout="soa", shared_w=SW)
    np.testing.assert_array_equal(a["params_bar"].cpu().numpy(), g["params_bar"].cpu().numpy())
    np.testing.assert_array_equal(a["shared_w_bar"].cpu().numpy(), g["shared_w_bar"].cpu().numpy())
