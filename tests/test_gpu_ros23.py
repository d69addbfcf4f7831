"""GPU parity of the Rosenbrock23 (second-order stiff) record, reverse sweep,
refresh and forward mode against the FP64 oracle, on the GPU's own exported
mesh (normwise relative error 1e-11 per trajectory vector, as for the other
FP64 methods), plus agreement of the GPU's and the oracle's own records.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2609_02876_gb300 import api, build
from paper_2609_02876_gb300 import workloads as W
from tests.test_gpu_tsit5 import assert_close, dev, record, reverse

pytestmark = pytest.mark.gpu
R23 = oracle.METHOD_ROSENBROCK23


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def oracle_on_mesh(wl, off, h, **kw):
    return oracle.replay_grad(wl["problem"], wl["params"], wl["y0"], wl["t0"], wl["t1"], wl["save_t"], off, h,
                              method=R23, **kw)


@pytest.mark.parametrize("name,n", [("robertson", 600), ("hires", 130)])
def test_ros23_record_and_reverse_match_oracle_on_gpu_mesh(name, n):
    wl = W.make(name, n)
    rec, ysv, st = record(wl, method="rosenbrock23")
    assert (st.cpu().numpy() == 0).all()
    g = reverse(rec, wl)
    off, h = rec.export_mesh()
    o = oracle_on_mesh(wl, off, h)
    assert o["ok"].all()
    assert_close(ysv.permute(2, 0, 1).cpu().numpy(), o["y_save"], "y_save")
    assert_close(g["loss"], o["loss"], "loss")
    assert_close(g["params_bar"].T, o["params_bar"], "params_bar")
    assert_close(g["y0_bar"].T, o["y0_bar"], "y0_bar")
    if name == "robertson":
        np.testing.assert_allclose(ysv.cpu().numpy().sum(1), 1.0, atol=1e-12)  # mass conservation


def test_ros23_mesh_agrees_with_oracle_record():
    """The same step rule on both sides; the FP32 controller factor moves h at
    ~1e-7 relative, so a trial near err = 1 can flip: most trajectories agree."""
    wl = W.make("robertson", 256)
    rec, _, _ = record(wl, method="rosenbrock23")
    off, h = rec.export_mesh()
    orec = oracle.record("robertson", wl["params"], wl["y0"], wl["t0"], wl["t1"], wl["save_t"], wl["rtol"],
                         wl["atol"], method=R23)
    same = np.diff(off) == orec["S"]
    assert same.mean() >= 0.8, same.mean()
    k = np.nonzero(same)[0][0]
    a, b = h[off[k]:off[k + 1]], orec["h"][orec["offsets"][k]:orec["offsets"][k + 1]]
    assert np.abs(a - b).max() / np.abs(b).max() < 1e-4


@pytest.mark.parametrize("k", [1, 3, 8])
def test_ros23_checkpoint_interval_and_linear_closed_form(k):
    rng = np.random.default_rng(8)
    n = 200
    A = np.array([[-40.0, 2.0, 1.0, -0.5]]) * (1 + 0.1 * rng.standard_normal((n, 4)))
    wl = dict(problem="linear", params=A, y0=rng.standard_normal((n, 2)), t0=0.0, t1=1.0,
              save_t=np.linspace(0.1, 1.0, 10), rtol=1e-6, atol=1e-9, w=None)
    rec, _, st = record(wl, method="rosenbrock23", ckpt_k=k)
    assert (st.cpu().numpy() == 0).all()
    g = reverse(rec, wl)
    off, h = rec.export_mesh()
    o = oracle_on_mesh(wl, off, h)
    assert_close(g["params_bar"].T, o["params_bar"], "params_bar")
    assert_close(g["y0_bar"].T, o["y0_bar"], "y0_bar")


def test_ros23_refresh_and_forward_mode():
    wl = W.make("robertson", 300)
    rec, _, _ = record(wl, method="rosenbrock23", want_saves=False)
    P, Y = dev(wl["params"].T), dev(wl["y0"].T)
    rv = api.reverse(rec, P, Y, layout="soa")
    fw = api.forward_grad(rec, P, Y, layout="soa")
    assert_close(fw["params_bar"].cpu().numpy().T, rv["params_bar"].cpu().numpy().T, "forward vs reverse")
    rng = np.random.default_rng(5)
    p1 = wl["params"] * (1 + 0.01 * rng.standard_normal(wl["params"].shape))
    api.refresh(rec, dev(p1.T), Y, layout="soa")
    g1 = api.reverse(rec, dev(p1.T), Y, layout="soa")
    off, h = rec.export_mesh()
    o = oracle.replay_grad("robertson", p1, wl["y0"], wl["t0"], wl["t1"], wl["save_t"], off, h, method=R23)
    assert_close(g1["params_bar"].cpu().numpy().T, o["params_bar"], "refreshed params_bar")


def test_ros23_solve_grad_and_forward_only_agree_with_record():
    wl = W.make("robertson", 257)
    rec, ysv, st = record(wl, method="rosenbrock23", step_counts=True)
    g = reverse(rec, wl)
    s = api.solve_grad("robertson", dev(wl["params"].T), dev(wl["y0"].T), wl["t0"], wl["t1"], wl["save_t"],
                       wl["rtol"], wl["atol"], layout="soa", method="rosenbrock23")
    np.testing.assert_allclose(s["params_bar"].cpu().numpy(), g["params_bar"], rtol=1e-13)
    f = api.solve("robertson", dev(wl["params"].T), dev(wl["y0"].T), wl["t0"], wl["t1"], wl["save_t"], wl["rtol"],
                  wl["atol"], layout="soa", method="rosenbrock23", step_counts=True)
    np.testing.assert_array_equal(f["y_save"].cpu().numpy(), ysv.cpu().numpy())
    np.testing.assert_array_equal(f["step_counts"].cpu().numpy(), rec.step_counts.cpu().numpy())


@pytest.mark.parametrize("name,n,stages", [("robertson", 700, 1), ("hires", 120, 0)])
def test_ros23_stored_stage_layout_is_bit_identical(name, n, stages):
    """gs_solve_grad keeps each Rosenbrock23 step's k1, u2 and LU of W when the
    segment fits (Robertson; not HIRES, d = 8) and rebuilds Y1 and the save
    states from them; its gradients equal the compact record's bit for bit."""
    wl = W.make(name, n)
    P, Y = dev(wl["params"].T), dev(wl["y0"].T)
    info = np.zeros(2, np.int32)
    s = api.solve_grad(name, P, Y, wl["t0"], wl["t1"], wl["save_t"], wl["rtol"], wl["atol"], layout="soa",
                       method="rosenbrock23", record_info=info)
    assert tuple(info) == (1, stages)
    rec, _, _ = record(wl, method="rosenbrock23", want_saves=False)
    g = api.reverse(rec, P, Y, layout="soa")
    np.testing.assert_array_equal(s["loss"].cpu().numpy(), g["loss"].cpu().numpy())
    np.testing.assert_array_equal(s["params_bar"].cpu().numpy(), g["params_bar"].cpu().numpy())
    np.testing.assert_array_equal(s["y0_bar"].cpu().numpy(), g["y0_bar"].cpu().numpy())
