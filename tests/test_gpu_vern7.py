"""GPU parity of the seventh-order Verner pair's record, reverse sweep and
refresh against the FP64 oracle, on the GPU's own exported mesh (normwise
relative error 1e-11 per trajectory vector, as for the other FP64 methods),
plus agreement of the GPU's and the oracle's own records and bit-equality of
the entry points that share the record.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2609_02876_gb300 import api, build
from paper_2609_02876_gb300 import workloads as W
from tests.test_gpu_tsit5 import assert_close, dev, record, reverse

pytestmark = pytest.mark.gpu
V7 = oracle.METHOD_VERNER7


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def oracle_on_mesh(wl, off, h, **kw):
    return oracle.replay_grad(wl["problem"], wl["params"], wl["y0"], wl["t0"], wl["t1"], wl["save_t"], off, h,
                              method=V7, **kw)


def linear_workload(n, seed=8):
    rng = np.random.default_rng(seed)
    A = np.array([[-0.5, 1.2, -1.7, -0.2]]) * (1 + 0.1 * rng.standard_normal((n, 4)))
    return dict(problem="linear", params=A, y0=rng.standard_normal((n, 2)), t0=0.0, t1=4.0,
                save_t=np.linspace(0.4, 4.0, 10), rtol=1e-8, atol=1e-10, w=None)


@pytest.mark.parametrize("name,n,rtol", [("lorenz", 512, None), ("lorenz", 300, 1e-10), ("vdp", 300, None),
                                         ("linear", 200, None)])
def test_vern7_record_and_reverse_match_oracle_on_gpu_mesh(name, n, rtol):
    wl = linear_workload(n) if name == "linear" else W.make(name, n)
    if rtol is not None:
        wl = dict(wl, rtol=rtol, atol=1e-2 * rtol)
    rec, ysv, st = record(wl, method="verner7")
    assert (st.cpu().numpy() == 0).all()
    g = reverse(rec, wl)
    off, h = rec.export_mesh()
    o = oracle_on_mesh(wl, off, h)
    assert o["ok"].all()
    assert_close(ysv.permute(2, 0, 1).cpu().numpy(), o["y_save"], "y_save")
    assert_close(g["loss"], o["loss"], "loss")
    assert_close(g["params_bar"].T, o["params_bar"], "params_bar")
    assert_close(g["y0_bar"].T, o["y0_bar"], "y0_bar")


def test_vern7_mesh_agrees_with_oracle_record():
    """The same step rule on both sides (controller exponent 1/7); the FP32
    controller factor moves h at ~1e-7 relative, so most trajectories agree."""
    wl = W.make("lorenz", 256)
    rec, _, _ = record(wl, method="verner7")
    off, h = rec.export_mesh()
    orec = oracle.record("lorenz", wl["params"], wl["y0"], wl["t0"], wl["t1"], wl["save_t"], wl["rtol"],
                         wl["atol"], method=V7)
    same = np.diff(off) == orec["S"]
    assert same.mean() >= 0.8, same.mean()
    k = np.nonzero(same)[0][0]
    a, b = h[off[k]:off[k + 1]], orec["h"][orec["offsets"][k]:orec["offsets"][k + 1]]
    assert np.abs(a - b).max() / np.abs(b).max() < 1e-4
    # seventh order: far fewer steps than Tsit5 on the same ensemble
    trec, _, _ = record(wl)
    assert np.diff(off).sum() < 0.8 * np.diff(trec.export_mesh()[0]).sum()


@pytest.mark.parametrize("k", [1, 3, 9])
def test_vern7_checkpoint_interval_and_user_cotangent(k):
    wl = W.make("vdp", 160)
    rec, ysv, st = record(wl, method="verner7", ckpt_k=k)
    assert (st.cpu().numpy() == 0).all()
    rng = np.random.default_rng(k)
    ybar = rng.standard_normal(ysv.shape)
    P, Y = dev(wl["params"].T), dev(wl["y0"].T)
    g = api.reverse(rec, P, Y, y_save_bar=torch.as_tensor(ybar, device="cuda"), layout="soa")
    off, h = rec.export_mesh()
    o = oracle_on_mesh(wl, off, h, ybar_save=np.ascontiguousarray(ybar.transpose(2, 0, 1)))
    assert_close(g["params_bar"].cpu().numpy().T, o["params_bar"], "params_bar")
    assert_close(g["y0_bar"].cpu().numpy().T, o["y0_bar"], "y0_bar")


def test_vern7_forward_mode_matches_oracle_and_reverse():
    """Forward mode over a Verner7 record: the directional derivatives equal the
    oracle's dual-number replay on the same mesh, and the forward-mode gradient
    equals the reverse sweep's (both to 1e-11 normwise)."""
    wl = W.make("lorenz", 400)
    rec, _, _ = record(wl, method="verner7", want_saves=False)
    P, Y = dev(wl["params"].T), dev(wl["y0"].T)
    rng = np.random.default_rng(21)
    pd = rng.standard_normal(wl["params"].shape) * wl["params"]
    yd = rng.standard_normal(wl["y0"].shape)
    j = api.replay_jvp(rec, P, Y, params_dot=dev(pd.T)[None], y0_dot=dev(yd.T)[None], layout="soa")
    off, h = rec.export_mesh()
    o = oracle.replay_jvp("lorenz", wl["params"], wl["y0"], wl["t0"], wl["t1"], wl["save_t"], off, h, pd, yd,
                          method=V7)
    ld = j["loss_dot"].cpu().numpy()[0]
    scale = np.abs(o["loss_dot"]).max()
    assert np.abs(ld - o["loss_dot"]).max() <= 1e-11 * scale
    fw = api.forward_grad(rec, P, Y, layout="soa")
    rv = api.reverse(rec, P, Y, layout="soa")
    assert_close(fw["params_bar"].cpu().numpy().T, rv["params_bar"].cpu().numpy().T, "forward vs reverse")
    assert_close(fw["y0_bar"].cpu().numpy().T, rv["y0_bar"].cpu().numpy().T, "forward vs reverse y0")


def test_vern7_refresh_at_new_parameters():
    wl = W.make("lorenz", 300)
    rec, _, _ = record(wl, method="verner7", want_saves=False)
    P, Y = dev(wl["params"].T), dev(wl["y0"].T)
    rng = np.random.default_rng(5)
    p1 = wl["params"] * (1 + 0.01 * rng.standard_normal(wl["params"].shape))
    api.refresh(rec, dev(p1.T), Y, layout="soa")
    g1 = api.reverse(rec, dev(p1.T), Y, layout="soa")
    off, h = rec.export_mesh()
    o = oracle.replay_grad("lorenz", p1, wl["y0"], wl["t0"], wl["t1"], wl["save_t"], off, h, method=V7)
    assert_close(g1["params_bar"].cpu().numpy().T, o["params_bar"], "refreshed params_bar")
    assert_close(g1["y0_bar"].cpu().numpy().T, o["y0_bar"], "refreshed y0_bar")


@pytest.mark.parametrize("name", ["lorenz", "vdp"])
def test_vern7_solve_grad_and_forward_only_agree_with_record(name):
    """gs_solve_grad stores the stage inputs (stored-stage layout) and reads
    them back in the reverse sweep; gs_forward_record keeps the compact record
    and recomputes them: the gradients agree bit for bit."""
    wl = W.make(name, 257)
    rec, ysv, st = record(wl, method="verner7", step_counts=True)
    g = reverse(rec, wl)
    info = np.zeros(2, np.int32)
    s = api.solve_grad(name, dev(wl["params"].T), dev(wl["y0"].T), wl["t0"], wl["t1"], wl["save_t"],
                       wl["rtol"], wl["atol"], layout="soa", method="verner7", record_info=info)
    assert tuple(info) == (1, 1)
    np.testing.assert_array_equal(s["params_bar"].cpu().numpy(), g["params_bar"])
    np.testing.assert_array_equal(s["y0_bar"].cpu().numpy(), g["y0_bar"])
    np.testing.assert_array_equal(s["loss"].cpu().numpy(), g["loss"])
    f = api.solve(name, dev(wl["params"].T), dev(wl["y0"].T), wl["t0"], wl["t1"], wl["save_t"], wl["rtol"],
                  wl["atol"], layout="soa", method="verner7", step_counts=True)
    np.testing.assert_array_equal(f["y_save"].cpu().numpy(), ysv.cpu().numpy())
    np.testing.assert_array_equal(f["step_counts"].cpu().numpy(), rec.step_counts.cpu().numpy())


def test_vern7_full_size_sample_is_bit_identical_and_matches_oracle():
    """n = 2^22: a random sample re-solved as its own ensemble reproduces the
    full-size gradients bit for bit; the sample matches the oracle on its mesh."""
    n, m = 1 << 22, 1024
    wl = W.make("lorenz", n)
    s = api.solve_grad("lorenz", dev(wl["params"].T), dev(wl["y0"].T), wl["t0"], wl["t1"], wl["save_t"], wl["rtol"],
                       wl["atol"], layout="soa", method="verner7")
    assert (s["status"] == 0).all().item()
    idx = np.sort(np.random.default_rng(3).choice(n, m, replace=False))
    full = {k: s[k].cpu().numpy()[..., idx] for k in ("loss", "params_bar", "y0_bar")}
    del s
    torch.cuda.empty_cache()
    ws = dict(wl, params=wl["params"][idx], y0=wl["y0"][idx])
    P, Y = dev(ws["params"].T), dev(ws["y0"].T)
    rec, _, _ = api.forward_record("lorenz", P, Y, ws["t0"], ws["t1"], ws["save_t"], ws["rtol"], ws["atol"],
                                   layout="soa", want_saves=False, method="verner7")
    g = api.reverse(rec, P, Y, layout="soa")
    np.testing.assert_array_equal(g["params_bar"].cpu().numpy(), full["params_bar"])
    np.testing.assert_array_equal(g["y0_bar"].cpu().numpy(), full["y0_bar"])
    off, h = rec.export_mesh()
    o = oracle_on_mesh(ws, off, h)
    assert_close(full["params_bar"].T, o["params_bar"], "params_bar")
    assert_close(full["y0_bar"].T, o["y0_bar"], "y0_bar")
