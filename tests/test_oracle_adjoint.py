"""Pins of the oracle's discrete adjoint (paper Sec. 3.1) on every problem.

1. Forward mode: a dual-number JVP of the same replay (the exact derivative of
   the same program, propagated in the other direction) must equal <grad, v>.
2. Central finite differences of the replay loss on the same recorded mesh,
   relative step 1e-6 along a seeded unit direction (paper Appendix B.6).
3. Shared weights of the LV UDE: brute-force finite differences on a
   2-trajectory ensemble.
"""
import numpy as np
import pytest

import oracle
from paper_2609_02876_gb300 import workloads as W

PROBS = ["lorenz", "vdp", "robertson", "hires", "lv_ude"]


def _setup(name, n):
    wl = W.make(name, n)
    rec = oracle.record(wl["problem"], wl["params"], wl["y0"], wl["t0"], wl["t1"], wl["save_t"], wl["rtol"],
                        wl["atol"], w=wl["w"])
    assert (rec["status"] == 0).all()
    return wl, rec


def _grad(wl, rec, params=None, y0=None, ybar=None, w=None):
    return oracle.replay_grad(wl["problem"], wl["params"] if params is None else params,
                              wl["y0"] if y0 is None else y0, wl["t0"], wl["t1"], wl["save_t"], rec["offsets"],
                              rec["h"], ybar_save=ybar, w=wl["w"] if w is None else w)


@pytest.mark.parametrize("name", PROBS)
def test_adjoint_equals_dual_number_jvp(name):
    wl, rec = _setup(name, 6)
    n, P = wl["params"].shape
    d = wl["y0"].shape[1]
    rng = np.random.default_rng(11)
    pdot = rng.standard_normal((n, P)) * wl["params"]  # relative directions
    ydot = rng.standard_normal((n, d))
    g = _grad(wl, rec)
    j = oracle.replay_jvp(wl["problem"], wl["params"], wl["y0"], wl["t0"], wl["t1"], wl["save_t"], rec["offsets"],
                          rec["h"], pdot, ydot, w=wl["w"])
    np.testing.assert_allclose(j["loss"], g["loss"], rtol=1e-15)
    lhs = (g["params_bar"] * pdot).sum(1) + (g["y0_bar"] * ydot).sum(1)
    scale = np.abs(g["params_bar"] * pdot).sum(1) + np.abs(g["y0_bar"] * ydot).sum(1)
    assert np.all(np.abs(lhs - j["loss_dot"]) <= 1e-12 * scale)
    # user cotangent of the save-time states
    ybar = rng.standard_normal(g["y_save"].shape)
    gu = _grad(wl, rec, ybar=ybar)
    lhs = (gu["params_bar"] * pdot).sum(1) + (gu["y0_bar"] * ydot).sum(1)
    rhs = (ybar * j["y_save_dot"]).sum((1, 2))
    scale = np.abs(gu["params_bar"] * pdot).sum(1) + np.abs(gu["y0_bar"] * ydot).sum(1)
    assert np.all(np.abs(lhs - rhs) <= 1e-12 * scale)


@pytest.mark.parametrize("name", PROBS)
def test_adjoint_matches_central_fd_on_same_mesh(name):
    wl, rec = _setup(name, 4)
    n, P = wl["params"].shape
    d = wl["y0"].shape[1]
    g = _grad(wl, rec)
    rng = np.random.default_rng(0)
    v = rng.standard_normal((n, P + d))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    x = np.concatenate([wl["params"], wl["y0"]], 1)
    eps = 1e-6 * np.maximum(np.abs(x), 1e-3)  # relative step 1e-6 per input
    dx = v * eps
    lp = _grad(wl, rec, params=(x + dx)[:, :P], y0=(x + dx)[:, P:])["loss"]
    lm = _grad(wl, rec, params=(x - dx)[:, :P], y0=(x - dx)[:, P:])["loss"]
    fd = (lp - lm) / 2.0
    ad = (np.concatenate([g["params_bar"], g["y0_bar"]], 1) * dx).sum(1)
    rel = np.abs(fd - ad) / np.maximum(np.abs(ad), 1e-300)
    assert rel.max() < 1e-5, rel


def test_ude_shared_weight_gradient_fd():
    wl, rec = _setup("lv_ude", 2)
    g = _grad(wl, rec)
    assert g["w_bar"].shape == (W.UDE_NW,)
    rng = np.random.default_rng(5)
    w0 = wl["w"]
    for trial in range(3):
        v = rng.standard_normal(w0.size)
        v /= np.linalg.norm(v)
        eps = 1e-6
        lp = _grad(wl, rec, w=w0 + eps * v)["loss"].sum()
        lm = _grad(wl, rec, w=w0 - eps * v)["loss"].sum()
        fd = (lp - lm) / (2 * eps)
        ad = g["w_bar"] @ v
        assert abs(fd - ad) <= 1e-6 * max(1.0, abs(ad)), (fd, ad)
    # biases of the output layer enter linearly: their gradient is exact in FD too
    assert np.abs(g["w_bar"]).max() > 0
