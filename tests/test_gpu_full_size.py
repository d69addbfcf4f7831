"""Parity at the full ensemble sizes, in the launch configuration the bench times.

Each trajectory's arithmetic does not depend on the rest of the ensemble (one
lane per trajectory, explicitly rounded operations, no cross-trajectory
reduction except the shared-weight sum). So a random sample of the full-size
ensemble, solved again as its own small ensemble, must reproduce the full-size
results bit for bit; the small run is then compared with the oracle on its
exported mesh, one trajectory at a time, within the usual FP64 bound.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2609_02876_gb300 import api, build
from paper_2609_02876_gb300 import workloads as W
from tests.test_gpu_tsit5 import FP32_MIXED_BOUND, assert_close, dev, fp32_mixed_errors

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def sub(wl, idx):
    return dict(wl, params=wl["params"][idx], y0=wl["y0"][idx])


@pytest.mark.parametrize("name,n,m,rtol", [("lorenz", 1 << 24, 2048, 1e-11), ("vdp", 1 << 20, 1024, 1e-11),
                                           ("robertson", 1 << 20, 1024, 1e-11), ("hires", 1 << 20, 256, 1e-11)])
def test_full_size_results_equal_their_sample_and_the_oracle(name, n, m, rtol):
    wl = W.make(name, n)
    s = api.solve_grad(name, dev(wl["params"].T), dev(wl["y0"].T), wl["t0"], wl["t1"], wl["save_t"], wl["rtol"],
                       wl["atol"], layout="soa")
    assert (s["status"] == 0).all().item()
    idx = np.sort(np.random.default_rng(3).choice(n, m, replace=False))
    full = {k: s[k].cpu().numpy()[..., idx] for k in ("loss", "params_bar", "y0_bar")}
    del s
    torch.cuda.empty_cache()
    ws = sub(wl, idx)
    P, Y = dev(ws["params"].T), dev(ws["y0"].T)
    rec, _, st = api.forward_record(name, P, Y, ws["t0"], ws["t1"], ws["save_t"], ws["rtol"], ws["atol"],
                                    layout="soa", want_saves=False)
    g = api.reverse(rec, P, Y, layout="soa")
    np.testing.assert_array_equal(g["loss"].cpu().numpy(), full["loss"])
    np.testing.assert_array_equal(g["params_bar"].cpu().numpy(), full["params_bar"])
    np.testing.assert_array_equal(g["y0_bar"].cpu().numpy(), full["y0_bar"])
    off, h = rec.export_mesh()
    o = oracle.replay_grad(name, ws["params"], ws["y0"], ws["t0"], ws["t1"], ws["save_t"], off, h)
    assert o["ok"].all()
    assert_close(full["loss"], o["loss"], "loss", rtol)
    assert_close(full["params_bar"].T, o["params_bar"], "params_bar", rtol)
    assert_close(full["y0_bar"].T, o["y0_bar"], "y0_bar", rtol)


def test_full_size_fp32_mixed_sample_and_oracle():
    """Lorenz at 2^24 in the FP32-mixed form (the bench's second line): a sample
    re-solved alone reproduces the full-size gradients bit for bit, and its error
    against the FP64 oracle on its mesh stays within the FP32-mixed bounds of the
    parity test (FP32_MIXED_BOUND)."""
    n, m = 1 << 24, 1024
    wl = W.make("lorenz", n)
    s = api.solve_grad("lorenz", dev(wl["params"].T), dev(wl["y0"].T), wl["t0"], wl["t1"], wl["save_t"], wl["rtol"],
                       wl["atol"], layout="soa", precision="fp32_mixed")
    assert (s["status"] == 0).all().item()
    idx = np.sort(np.random.default_rng(5).choice(n, m, replace=False))
    full = {k: s[k].cpu().numpy()[..., idx] for k in ("params_bar", "y0_bar")}
    del s
    torch.cuda.empty_cache()
    ws = sub(wl, idx)
    P, Y = dev(ws["params"].T), dev(ws["y0"].T)
    rec, _, _ = api.forward_record("lorenz", P, Y, ws["t0"], ws["t1"], ws["save_t"], ws["rtol"], ws["atol"],
                                   layout="soa", want_saves=False, precision="fp32_mixed")
    g = api.reverse(rec, P, Y, layout="soa")
    np.testing.assert_array_equal(g["params_bar"].cpu().numpy(), full["params_bar"])
    np.testing.assert_array_equal(g["y0_bar"].cpu().numpy(), full["y0_bar"])
    off, h = rec.export_mesh()
    o = oracle.replay_grad("lorenz", ws["params"], ws["y0"], ws["t0"], ws["t1"], ws["save_t"], off, h)
    e = fp32_mixed_errors(full["params_bar"].T, full["y0_bar"].T, o)
    med, mx = FP32_MIXED_BOUND["lorenz"]
    assert np.median(e) <= med and e.max() <= mx, (np.median(e), e.max())


def test_full_size_ude_sample_and_oracle():
    """LV UDE at 2^18 (FP32 network): per-trajectory results of a sample equal the
    full run bit for bit and match the FP64 oracle within the FP32 bound 1e-4."""
    n, m = 1 << 18, 512
    wl = W.make("lv_ude", n)
    SW = torch.as_tensor(np.asarray(wl["w"], dtype=np.float32), device="cuda")
    s = api.solve_grad("lv_ude", dev(wl["params"].T), dev(wl["y0"].T), wl["t0"], wl["t1"], wl["save_t"],
                       wl["rtol"], wl["atol"], layout="soa", shared_w=SW, precision="fp32_mixed")
    idx = np.sort(np.random.default_rng(4).choice(n, m, replace=False))
    full = {k: s[k].cpu().numpy()[..., idx] for k in ("params_bar", "y0_bar")}
    ws = sub(wl, idx)
    P, Y = dev(ws["params"].T), dev(ws["y0"].T)
    rec, _, _ = api.forward_record("lv_ude", P, Y, ws["t0"], ws["t1"], ws["save_t"], ws["rtol"], ws["atol"],
                                   layout="soa", want_saves=False, shared_w=SW, precision="fp32_mixed")
    g = api.reverse(rec, P, Y, layout="soa", shared_w=SW)
    np.testing.assert_array_equal(g["params_bar"].cpu().numpy(), full["params_bar"])
    np.testing.assert_array_equal(g["y0_bar"].cpu().numpy(), full["y0_bar"])
    off, h = rec.export_mesh()
    o = oracle.replay_grad("lv_ude", ws["params"], ws["y0"], ws["t0"], ws["t1"], ws["save_t"], off, h,
                           w=SW.cpu().numpy().astype(np.float64))
    assert_close(full["params_bar"].T, o["params_bar"], "params_bar", 1e-4)
    assert_close(full["y0_bar"].T, o["y0_bar"], "y0_bar", 1e-4)
