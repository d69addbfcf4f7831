"""GPU parity of the LV UDE (shared-weight MLP 2-16-16-2) record + reverse sweep.

The GPU runs the network and the state in FP32 (control in FP64) with the
shared-weight gradient accumulated by tensor-core MMAs (3xTF32); the reference
is the oracle's FP64 network with the same (FP32-rounded) weights, replayed on
the GPU's own mesh. Tolerance derived from FP32 arithmetic: the per-step
rounding (6e-8) carried through ~32 steps of 6 stages and two tanh layers
stays below 1e-4 normwise for the per-trajectory gradients and for the
ensemble-summed weight gradient.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2609_02876_gb300 import api, build, shard
from paper_2609_02876_gb300 import workloads as W
from tests.test_gpu_tsit5 import assert_close, dev

pytestmark = pytest.mark.gpu
TOL = 1e-4


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def _setup(n):
    wl = W.make("lv_ude", n)
    w32 = wl["w"].astype(np.float32)
    wl = dict(wl, w=w32.astype(np.float64))
    return wl, torch.as_tensor(w32, device="cuda")


def _record(wl, w, **kw):
    return api.forward_record("lv_ude", dev(wl["params"].T), dev(wl["y0"].T), wl["t0"], wl["t1"], wl["save_t"],
                              wl["rtol"], wl["atol"], shared_w=w, layout="soa", precision="fp32_mixed", **kw)


def _reverse(rec, wl, w, ybar=None):
    g = api.reverse(rec, dev(wl["params"].T), dev(wl["y0"].T), y_save_bar=ybar, shared_w=w, layout="soa")
    return {k: (v.cpu().numpy() if v is not None else None) for k, v in g.items()}


@pytest.mark.parametrize("n", [1000, 4097])
def test_ude_gradients_match_fp64_oracle_on_gpu_mesh(n):
    wl, w = _setup(n)
    rec, ysv, st = _record(wl, w)
    assert (st.cpu().numpy() == 0).all()
    g = _reverse(rec, wl, w)
    off, h = rec.export_mesh()
    o = oracle.replay_grad("lv_ude", wl["params"], wl["y0"], wl["t0"], wl["t1"], wl["save_t"], off, h, w=wl["w"])
    assert o["ok"].all()
    assert_close(ysv.permute(2, 0, 1).cpu().numpy(), o["y_save"], "y_save", rtol=TOL)
    assert_close(g["params_bar"].T, o["params_bar"], "params_bar (a, d)", rtol=TOL)
    assert_close(g["y0_bar"].T, o["y0_bar"], "y0_bar", rtol=TOL)
    wb, wo = g["shared_w_bar"].astype(np.float64), o["w_bar"]
    err = np.abs(wb - wo).max() / np.abs(wo).max()
    assert err < TOL, f"shared-weight gradient: normwise rel err {err:.3e}"


def test_ude_weight_gradient_is_deterministic_and_solve_grad_agrees():
    wl, w = _setup(2048)
    rec, _, _ = _record(wl, w, want_saves=False)
    g1 = _reverse(rec, wl, w)
    g2 = _reverse(rec, wl, w)
    np.testing.assert_array_equal(g1["shared_w_bar"], g2["shared_w_bar"])
    np.testing.assert_array_equal(g1["params_bar"], g2["params_bar"])
    s = api.solve_grad("lv_ude", dev(wl["params"].T), dev(wl["y0"].T), wl["t0"], wl["t1"], wl["save_t"],
                       wl["rtol"], wl["atol"], shared_w=w, layout="soa", precision="fp32_mixed")
    np.testing.assert_array_equal(s["shared_w_bar"].cpu().numpy(), g1["shared_w_bar"])
    np.testing.assert_array_equal(s["params_bar"].cpu().numpy(), g1["params_bar"])


def test_ude_user_cotangent():
    wl, w = _setup(512)
    rec, _, _ = _record(wl, w)
    rng = np.random.default_rng(8)
    ybar = rng.standard_normal((512, len(wl["save_t"]), 2))
    g = _reverse(rec, wl, w, ybar=dev(ybar.transpose(1, 2, 0)))
    off, h = rec.export_mesh()
    o = oracle.replay_grad("lv_ude", wl["params"], wl["y0"], wl["t0"], wl["t1"], wl["save_t"], off, h, w=wl["w"],
                           ybar_save=ybar)
    assert_close(g["params_bar"].T, o["params_bar"], "params_bar", rtol=TOL)
    err = np.abs(g["shared_w_bar"] - o["w_bar"]).max() / np.abs(o["w_bar"]).max()
    assert err < TOL, err


def test_autograd_returns_the_shared_weight_gradient():
    """odeint_ensemble with the network weights as a differentiable input: a
    user loss on the save states, backward through gs_reverse, gives the
    per-trajectory (a, d) and y0 gradients and the ensemble-summed weight
    gradient of the oracle's adjoint of the same loss on the GPU's mesh."""
    wl, w = _setup(384)
    p = dev(wl["params"]).requires_grad_(True)
    y0 = dev(wl["y0"]).requires_grad_(True)
    wr = w.clone().requires_grad_(True)
    ysv = api.odeint_ensemble("lv_ude", p, y0, wl["t0"], wl["t1"], wl["save_t"], wl["rtol"], wl["atol"],
                              shared_w=wr, precision="fp32_mixed")
    target = torch.linspace(0.5, 1.5, ysv.numel(), dtype=torch.float64, device="cuda").reshape(ysv.shape)
    loss = ((ysv - target) ** 2).sum()
    loss.backward()
    assert wr.grad is not None and wr.grad.dtype == torch.float32 and wr.grad.shape == w.shape
    cot = 2 * (ysv.detach() - target).cpu().numpy()
    rec, _, _ = _record(wl, w)
    off, h = rec.export_mesh()
    o = oracle.replay_grad("lv_ude", wl["params"], wl["y0"], wl["t0"], wl["t1"], wl["save_t"], off, h, w=wl["w"],
                           ybar_save=cot)
    assert_close(p.grad.cpu().numpy(), o["params_bar"], "params_bar", rtol=TOL)
    assert_close(y0.grad.cpu().numpy(), o["y0_bar"], "y0_bar", rtol=TOL)
    err = np.abs(wr.grad.cpu().numpy() - o["w_bar"]).max() / np.abs(o["w_bar"]).max()
    assert err < TOL, err


def test_sharded_weight_gradient_equals_unsharded():
    """The multi-GPU partition of the UDE ensemble run as 4 shards one after another
    on this GPU: each shard's gs_solve_grad weight gradient (FP32), added in shard
    order in FP64 as the ranks' reduction does, equals the unsharded one to the
    rounding of the FP32 results (each shard's sum and the whole one carry a
    relative error of a few 1e-7 of the largest entry; bound 2e-6)."""
    n = 6000
    wl, w = _setup(n)
    P, Y = dev(wl["params"].T), dev(wl["y0"].T)
    whole = api.solve_grad("lv_ude", P, Y, wl["t0"], wl["t1"], wl["save_t"], wl["rtol"], wl["atol"], shared_w=w,
                           layout="soa", precision="fp32_mixed")
    parts, pbar = [], []
    for r in range(4):
        lo, hi = shard.shard_range(n, r, 4)
        s = api.solve_grad("lv_ude", P[:, lo:hi].contiguous(), Y[:, lo:hi].contiguous(), wl["t0"], wl["t1"],
                           wl["save_t"], wl["rtol"], wl["atol"], shared_w=w, layout="soa", precision="fp32_mixed")
        parts.append(s["shared_w_bar"].cpu().numpy())
        pbar.append(s["params_bar"].cpu().numpy())
    # per-trajectory gradients do not depend on the partition
    np.testing.assert_array_equal(np.concatenate(pbar, 1), whole["params_bar"].cpu().numpy())
    summed = shard.sum_in_rank_order(parts)
    ref = whole["shared_w_bar"].cpu().numpy().astype(np.float64)
    err = np.abs(summed - ref).max() / np.abs(ref).max()
    assert err < 2e-6, err
