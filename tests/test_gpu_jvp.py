"""GPU forward mode of the replay (gs_replay_jvp, gs_forward_grad) against the
FP64 oracle's dual-number replay on the GPU's own recorded mesh.

A directional derivative dL = sum_q g_q v_q can cancel, so its error is
measured against the condition scale sum_q |g_q v_q| (g the oracle's
gradient): |dL_gpu - dL_oracle| <= 1e-11 * scale. Save-state tangents are
compared normwise per trajectory (all saves and components of one direction
form one vector), as for the other FP64 parity tests.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2609_02876_gb300 import api, build
from paper_2609_02876_gb300 import workloads as W
from tests.test_gpu_tsit5 import assert_close, dev, record

pytestmark = pytest.mark.gpu
RTOL = 1e-11


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def directions(wl, nd, seed):
    rng = np.random.default_rng(seed)
    n, P = wl["params"].shape
    d = wl["y0"].shape[1]
    pd = rng.standard_normal((nd, n, P)) * np.abs(wl["params"])[None]  # relative perturbations of theta
    yd = rng.standard_normal((nd, n, d)) * np.maximum(np.abs(wl["y0"]), 1e-3)[None]
    return pd, yd


@pytest.mark.parametrize("name,n,nd", [("lorenz", 700, 4), ("vdp", 333, 2), ("robertson", 257, 3), ("hires", 65, 1)])
def test_replay_jvp_matches_oracle_on_gpu_mesh(name, n, nd):
    wl = W.make(name, n)
    rec, _, st = record(wl, want_saves=False)
    assert (st.cpu().numpy() == 0).all()
    pd, yd = directions(wl, nd, 5)
    g = api.replay_jvp(rec, dev(wl["params"]), dev(wl["y0"]), dev(pd), dev(yd), want_y_save_dot=True)
    off, h = rec.export_mesh()
    ograd = oracle.replay_grad(name, wl["params"], wl["y0"], wl["t0"], wl["t1"], wl["save_t"], off, h)
    assert_close(g["loss"].cpu().numpy(), ograd["loss"], "loss")
    ldot = g["loss_dot"].cpu().numpy()
    ysd = g["y_save_dot"].cpu().numpy()
    for q in range(nd):
        o = oracle.replay_jvp(name, wl["params"], wl["y0"], wl["t0"], wl["t1"], wl["save_t"], off, h, pd[q], yd[q])
        scale = (np.abs(ograd["params_bar"] * pd[q]).sum(1) + np.abs(ograd["y0_bar"] * yd[q]).sum(1))
        err = np.abs(ldot[q] - o["loss_dot"]) / scale
        assert err.max() <= RTOL, f"loss_dot dir {q}: {err.max():.3e}"
        assert_close(ysd[q].reshape(n, -1), o["y_save_dot"].reshape(n, -1), f"y_save_dot dir {q}")


@pytest.mark.parametrize("name", ["lorenz", "vdp", "robertson", "hires"])
def test_forward_grad_equals_reverse_gradient(name):
    """Forward mode along the unit directions and the reverse sweep are two
    evaluations of the same derivative of the same replay."""
    wl = W.make(name, 300)
    rec, _, _ = record(wl, want_saves=False)
    P, Y = dev(wl["params"].T), dev(wl["y0"].T)
    rv = api.reverse(rec, P, Y, layout="soa")
    fw = api.forward_grad(rec, P, Y, layout="soa")
    assert_close(fw["loss"].cpu().numpy(), rv["loss"].cpu().numpy(), "loss")
    assert_close(fw["params_bar"].cpu().numpy().T, rv["params_bar"].cpu().numpy().T, "params_bar")
    assert_close(fw["y0_bar"].cpu().numpy().T, rv["y0_bar"].cpu().numpy().T, "y0_bar")
    only_p = api.forward_grad(rec, P, Y, wrt=("params",), layout="soa")
    assert only_p["y0_bar"] is None
    np.testing.assert_array_equal(only_p["params_bar"].cpu().numpy(), fw["params_bar"].cpu().numpy())


def test_linear_forward_grad_both_methods_match_closed_form_adjoint():
    wl = W.make("lorenz", 8)  # only for t0, t1 and the save times
    rng = np.random.default_rng(3)
    n = 96
    A = rng.standard_normal((n, 4)) * 0.5
    y0 = rng.standard_normal((n, 2))
    lw = dict(problem="linear", params=A, y0=y0, t0=0.0, t1=1.0, save_t=wl["save_t"], rtol=1e-8, atol=1e-10, w=None)
    for method in ("tsit5", "rodas5p"):
        rec, _, _ = record(lw, want_saves=False, method=method)
        P, Y = dev(A.T), dev(y0.T)
        fw = api.forward_grad(rec, P, Y, layout="soa")
        off, h = rec.export_mesh()
        o = oracle.replay_grad("linear", A, y0, 0.0, 1.0, wl["save_t"], off, h,
                               method=oracle.METHOD_TSIT5 if method == "tsit5" else oracle.METHOD_RODAS5P)
        assert_close(fw["params_bar"].cpu().numpy().T, o["params_bar"], f"params_bar {method}")
        assert_close(fw["y0_bar"].cpu().numpy().T, o["y0_bar"], f"y0_bar {method}")


def test_directions_are_independent_of_their_launch_grouping():
    """Four directions run as launches of 3 + 1; each equals its own one-direction call bit for bit."""
    wl = W.make("lorenz", 512)
    rec, _, _ = record(wl, want_saves=False)
    pd, yd = directions(wl, 4, 9)
    P, Y = dev(wl["params"]), dev(wl["y0"])
    allg = api.replay_jvp(rec, P, Y, dev(pd), dev(yd), want_y_save_dot=True)
    for q in range(4):
        one = api.replay_jvp(rec, P, Y, dev(pd[q]), dev(yd[q]), want_y_save_dot=True)
        np.testing.assert_array_equal(one["loss_dot"].cpu().numpy()[0], allg["loss_dot"].cpu().numpy()[q])
        np.testing.assert_array_equal(one["y_save_dot"].cpu().numpy()[0], allg["y_save_dot"].cpu().numpy()[q])


def test_zero_tangent_inputs_and_failed_trajectories():
    wl = W.make("vdp", 96)
    p = wl["params"].copy()
    p[11, 0] = np.nan
    rec, _, st = record(dict(wl, params=p), want_saves=False, check=False)
    assert st.cpu().numpy()[11] == 3
    rng = np.random.default_rng(2)
    yd = rng.standard_normal((96, 2))
    g = api.replay_jvp(rec, dev(p), dev(wl["y0"]), None, dev(yd))
    ld = g["loss_dot"].cpu().numpy()[0]
    assert np.isnan(ld[11]) and np.isfinite(np.delete(ld, 11)).all()
    off, h = rec.export_mesh()
    keep = np.delete(np.arange(96), 11)
    sub_off = np.concatenate([[0], np.cumsum(np.diff(off)[keep])])
    sub_h = np.concatenate([h[off[k]:off[k + 1]] for k in keep])
    o = oracle.replay_jvp("vdp", p[keep], wl["y0"][keep], wl["t0"], wl["t1"], wl["save_t"], sub_off, sub_h,
                          np.zeros((95, 1)), yd[keep])
    ograd = oracle.replay_grad("vdp", p[keep], wl["y0"][keep], wl["t0"], wl["t1"], wl["save_t"], sub_off, sub_h)
    scale = np.abs(ograd["y0_bar"] * yd[keep]).sum(1)
    assert (np.abs(ld[keep] - o["loss_dot"]) / scale).max() <= RTOL
