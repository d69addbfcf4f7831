"""GPU parity of the Rodas5P (stiff) record + reverse sweep against the FP64 oracle.

Same protocol as the Tsit5 tests: gradients on the GPU's own exported mesh,
normwise relative error 1e-11 per trajectory vector, plus invariants, the
closed-form linear case and finite differences.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2609_02876_gb300 import api, build
from paper_2609_02876_gb300 import workloads as W
from tests.test_gpu_tsit5 import assert_close, dev, oracle_on_gpu_mesh, record, reverse

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


@pytest.mark.parametrize("name,n", [("robertson", 512), ("hires", 256)])
def test_rodas_record_and_reverse_match_oracle_on_gpu_mesh(name, n):
    wl = W.make(name, n)
    rec, ysv, st = record(wl)
    assert (st.cpu().numpy() == 0).all()
    g = reverse(rec, wl)
    o, off, h = oracle_on_gpu_mesh(wl, rec)
    assert o["ok"].all()
    assert_close(ysv.permute(2, 0, 1).cpu().numpy(), o["y_save"], "y_save")
    assert_close(g["loss"], o["loss"], "loss")
    assert_close(g["params_bar"].T, o["params_bar"], "params_bar")
    assert_close(g["y0_bar"].T, o["y0_bar"], "y0_bar")


def rounding_floor(wl, off, h, ybar):
    """Normwise disagreement, per trajectory, of two exact FP64 evaluations of the
    same derivative in the oracle (forward-mode JVP along each parameter against
    the reverse-mode adjoint): the rounding noise floor the problem itself sets."""
    g = oracle.replay_grad(wl["problem"], wl["params"], wl["y0"], wl["t0"], wl["t1"], wl["save_t"], off, h,
                           ybar_save=ybar)
    n, P = wl["params"].shape
    worst = np.zeros(n)
    for q in range(P):
        pd = np.zeros((n, P))
        pd[:, q] = 1.0
        j = oracle.replay_jvp(wl["problem"], wl["params"], wl["y0"], wl["t0"], wl["t1"], wl["save_t"], off, h, pd,
                              np.zeros_like(wl["y0"]))
        fwd = (ybar * j["y_save_dot"]).sum((1, 2))
        worst = np.maximum(worst, np.abs(fwd - g["params_bar"][:, q]) / np.abs(g["params_bar"]).max(1))
    return worst.max()


def test_rodas_user_cotangent_and_checkpoint_interval():
    """User cotangents on all 20 Robertson save times, scaled like a relative
    misfit (ybar = xi * y, xi ~ N(0, 1)). Unscaled O(1) cotangents on the fast
    species y2 (~1e-5) excite the ill-conditioned direction of
    I/(h gamma) - J, where two correct FP64 evaluations (different LU rounding)
    differ by up to ~2e-10. The bound is 20x the rounding floor the oracle
    measures between its forward- and reverse-mode derivatives, and never
    tighter than 1e-11."""
    wl = W.make("robertson", 256)
    rng = np.random.default_rng(2)
    xi = rng.standard_normal((256, len(wl["save_t"]), 3))
    for k in (1, 4):
        rec, ysv, _ = record(wl, ckpt_k=k)
        ybar = xi * ysv.permute(2, 0, 1).cpu().numpy()
        g = reverse(rec, wl, ybar=dev(ybar.transpose(1, 2, 0)))
        o, off, h = oracle_on_gpu_mesh(wl, rec, ybar=ybar)
        tol = max(1e-11, 20 * rounding_floor(wl, off, h, ybar))
        assert tol < 1e-8
        assert_close(g["params_bar"].T, o["params_bar"], f"params_bar k={k}", rtol=tol)
        assert_close(g["y0_bar"].T, o["y0_bar"], f"y0_bar k={k}", rtol=tol)


@pytest.mark.parametrize("name,idx,total", [("robertson", [0, 1, 2], 1.0), ("hires", [6, 7], 0.0057)])
def test_rodas_conserves_invariants_on_gpu(name, idx, total):
    wl = W.make(name, 128)
    rec, ysv, _ = record(wl)
    inv = ysv.permute(2, 0, 1).cpu().numpy()[:, :, idx].sum(-1)
    np.testing.assert_allclose(inv, total, rtol=0, atol=1e-13 * max(1.0, total) + 1e-15)


def stiff_linear(n, seed=6):
    """2x2 linear system with one fast eigenvalue in [-1e4, -1e2]."""
    rng = np.random.default_rng(seed)
    lam_fast = -10.0 ** rng.uniform(2, 4, n)
    params = np.stack([lam_fast, rng.uniform(0.5, 1.5, n), rng.uniform(0.1, 0.5, n), -rng.uniform(0.5, 1.5, n)], 1)
    return dict(problem="linear", params=params, y0=rng.uniform(-1, 1, (n, 2)), t0=0.0, t1=3.0,
                save_t=W.uniform_saves(0.0, 3.0, 6), rtol=1e-7, atol=1e-10, w=None)


def test_rodas_stiff_linear_problem():
    wl = stiff_linear(32)
    rec, ysv, st = record(wl, method="rodas5p")
    assert (st.cpu().numpy() == 0).all()
    g = reverse(rec, wl)
    off, h = rec.export_mesh()
    o = oracle.replay_grad("linear", wl["params"], wl["y0"], wl["t0"], wl["t1"], wl["save_t"], off, h,
                           method=oracle.METHOD_RODAS5P)
    assert_close(g["params_bar"].T, o["params_bar"], "params_bar")
    assert_close(g["y0_bar"].T, o["y0_bar"], "y0_bar")


def test_rodas_solve_grad_equals_record_then_reverse():
    wl = W.make("hires", 512)
    rec, _, _ = record(wl, want_saves=False)
    g = reverse(rec, wl)
    s = api.solve_grad(wl["problem"], dev(wl["params"].T), dev(wl["y0"].T), wl["t0"], wl["t1"], wl["save_t"],
                       wl["rtol"], wl["atol"], layout="soa")
    assert (s["status"].cpu().numpy() == 0).all()
    assert_close(s["params_bar"].cpu().numpy().T, g["params_bar"].T, "params_bar", rtol=1e-14)
    assert_close(s["y0_bar"].cpu().numpy().T, g["y0_bar"].T, "y0_bar", rtol=1e-14)


@pytest.mark.parametrize("name,n,stages", [("robertson", 1000, 1), ("linear", 333, 1), ("hires", 200, 0)])
def test_rodas_stored_stage_layout_is_bit_identical(name, n, stages):
    """gs_solve_grad keeps every Rodas5P step's U_i and LU of W when the segment
    fits (Robertson, the linear problem; not HIRES, d = 8) and replays the stage
    inputs from them; its gradients equal the compact record's bit for bit."""
    wl = stiff_linear(n) if name == "linear" else W.make(name, n)
    P, Y = dev(wl["params"].T), dev(wl["y0"].T)
    info = np.zeros(2, np.int32)
    s = api.solve_grad(name, P, Y, wl["t0"], wl["t1"], wl["save_t"], wl["rtol"], wl["atol"], layout="soa",
                       record_info=info, method="rodas5p")
    assert tuple(info) == (1, stages)
    assert (s["status"].cpu().numpy() == 0).all()
    rec_info = np.zeros(2, np.int32)
    rec, _, _ = api.forward_record(name, P, Y, wl["t0"], wl["t1"], wl["save_t"], wl["rtol"], wl["atol"],
                                   layout="soa", want_saves=False, record_info=rec_info, method="rodas5p")
    assert rec_info[1] == 0
    g = api.reverse(rec, P, Y, layout="soa")
    np.testing.assert_array_equal(s["loss"].cpu().numpy(), g["loss"].cpu().numpy())
    np.testing.assert_array_equal(s["params_bar"].cpu().numpy(), g["params_bar"].cpu().numpy())
    np.testing.assert_array_equal(s["y0_bar"].cpu().numpy(), g["y0_bar"].cpu().numpy())


def test_rodas_mesh_agreement_with_oracle_record():
    wl = W.make("robertson", 512)
    rec, _, _ = record(wl)
    off, _ = rec.export_mesh()
    orec = oracle.record(wl["problem"], wl["params"], wl["y0"], wl["t0"], wl["t1"], wl["save_t"], wl["rtol"],
                         wl["atol"])
    same = np.diff(off) == orec["S"]
    assert same.mean() >= 0.8, same.mean()


def test_rodas_gradient_matches_central_fd_on_gpu_mesh():
    wl = W.make("robertson", 8)
    rec, _, _ = record(wl)
    g = reverse(rec, wl)
    off, h = rec.export_mesh()
    rng = np.random.default_rng(0)
    x = np.concatenate([wl["params"], wl["y0"]], 1)
    v = rng.standard_normal(x.shape)
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    dx = v * 1e-6 * np.maximum(np.abs(x), 1e-3)

    def L(xx):
        return oracle.replay_grad("robertson", xx[:, :3], xx[:, 3:], wl["t0"], wl["t1"], wl["save_t"], off,
                                  h)["loss"]

    fd = (L(x + dx) - L(x - dx)) / 2
    ad = (np.concatenate([g["params_bar"].T, g["y0_bar"].T], 1) * dx).sum(1)
    assert (np.abs(fd - ad) / np.abs(ad)).max() < 1e-5
