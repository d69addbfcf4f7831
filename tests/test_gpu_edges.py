"""Degenerate and maximum cases of the GPU path, each against the FP64 oracle on
the GPU's own mesh (normwise relative error 1e-11 per trajectory vector)."""
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


def check(wl, method=None, **opts):
    P, Y = dev(wl["params"].T), dev(wl["y0"].T)
    rec, ysv, st = api.forward_record(wl["problem"], P, Y, wl["t0"], wl["t1"], wl["save_t"], wl["rtol"],
                                      wl["atol"], layout="soa", method=method, **opts)
    assert (st.cpu().numpy() == 0).all()
    g = api.reverse(rec, P, Y, layout="soa")
    off, h = rec.export_mesh()
    om = {None: oracle.METHOD_AUTO, "rosenbrock23": oracle.METHOD_ROSENBROCK23,
          "verner7": oracle.METHOD_VERNER7}[method]
    o = oracle.replay_grad(wl["problem"], wl["params"], wl["y0"], wl["t0"], wl["t1"], wl["save_t"], off, h,
                           method=om)
    assert_close(ysv.permute(2, 0, 1).cpu().numpy(), o["y_save"], "y_save")
    assert_close(g["params_bar"].cpu().numpy().T, o["params_bar"], "params_bar")
    assert_close(g["y0_bar"].cpu().numpy().T, o["y0_bar"], "y0_bar")
    return off, h


def test_span_of_a_single_step():
    """t1 - t0 = 1e-7: the starting step is clamped to the span, one accepted step;
    the save at t1 is the step's end state."""
    wl = dict(W.make("lorenz", 100), t1=1e-7, save_t=np.array([5e-8, 1e-7]))
    off, h = check(wl)
    assert (np.diff(off) == 1).all()
    np.testing.assert_allclose(h, 1e-7, rtol=1e-15)


def test_maximum_number_of_save_times():
    wl = W.make("vdp", 300)
    wl = dict(wl, save_t=np.linspace(0.0, wl["t1"], 257)[1:])  # 256 saves, t1 included
    check(wl)


def test_saves_before_the_first_step_ends_and_close_to_t0():
    wl = W.make("lorenz", 64)
    wl = dict(wl, save_t=np.array([1e-12, 1e-9, 1e-6, 0.5, 1.0]))
    check(wl)


def test_user_first_step_and_loose_tolerance():
    wl = dict(W.make("lorenz", 128), rtol=1e-2, atol=1e-4)
    off, h = check(wl, h0=1e-3)
    first = h[off[:-1]]
    assert np.all(first <= 1e-3)  # the given step is the first trial (accepted or shrunk)


@pytest.mark.parametrize("name,method", [("lorenz", None), ("robertson", None), ("robertson", "rosenbrock23"),
                                         ("vdp", "verner7")])
def test_single_trajectory_through_every_entry_point(name, method):
    wl = W.make(name, 1)
    check(wl, method=method)
    P, Y = dev(wl["params"].T), dev(wl["y0"].T)
    s = api.solve_grad(name, P, Y, wl["t0"], wl["t1"], wl["save_t"], wl["rtol"], wl["atol"], layout="soa",
                       method=method)
    f = api.solve(name, P, Y, wl["t0"], wl["t1"], wl["save_t"], wl["rtol"], wl["atol"], layout="soa",
                  method=method)
    rec, ysv, _ = api.forward_record(name, P, Y, wl["t0"], wl["t1"], wl["save_t"], wl["rtol"], wl["atol"],
                                     layout="soa", method=method)
    np.testing.assert_array_equal(f["y_save"].cpu().numpy(), ysv.cpu().numpy())
    fg = api.forward_grad(rec, P, Y, layout="soa")
    assert_close(fg["params_bar"].cpu().numpy().T, s["params_bar"].cpu().numpy().T, "forward vs reverse")
    hs = api.solve_grad_host(name, torch.from_numpy(np.ascontiguousarray(wl["params"].T)),
                             torch.from_numpy(np.ascontiguousarray(wl["y0"].T)), wl["t0"], wl["t1"], wl["save_t"],
                             wl["rtol"], wl["atol"], method=method)
    np.testing.assert_array_equal(hs["params_bar"].numpy(), s["params_bar"].cpu().numpy())


def test_empty_ensembles_are_no_ops():
    z = torch.empty((3, 0), dtype=torch.float64, device="cuda")
    wl = W.make("lorenz", 1)
    s = api.solve_grad("lorenz", z, z, 0.0, 1.0, wl["save_t"], 1e-6, 1e-8, layout="soa")
    assert s["params_bar"].shape == (3, 0)
    f = api.solve("lorenz", z, z, 0.0, 1.0, wl["save_t"], 1e-6, 1e-8, layout="soa")
    assert f["y_final"].shape == (3, 0)
    e = torch.empty((3, 0), dtype=torch.float64)
    h = api.solve_grad_host("lorenz", e, e, 0.0, 1.0, wl["save_t"], 1e-6, 1e-8)
    assert h["params_bar"].shape == (3, 0)


def test_record_outgrowing_the_first_arena_guess():
    """A lightly damped 2x2 rotation over 16 periods: several times the steps the
    first arena size assumes, so the record kernel overflows its arena, the host
    regrows it to the measured demand and reruns; the results still match the
    oracle, and the stored-stage workspace (gs_solve_grad) agrees with the
    compact record. (A linear, non-chaotic system: rounding differences between
    the two sides do not grow exponentially over the long span.)"""
    n = 2000
    rng = np.random.default_rng(12)
    A = np.array([[-0.01, 1.0, -1.0, -0.01]]) * (1 + 0.05 * rng.standard_normal((n, 4)))
    wl = dict(problem="linear", params=A, y0=rng.standard_normal((n, 2)), t0=0.0, t1=100.0,
              save_t=np.linspace(10.0, 100.0, 10), rtol=1e-8, atol=1e-10, w=None)
    off, h = check(wl)
    assert np.diff(off).mean() > 300
    P, Y = dev(wl["params"].T), dev(wl["y0"].T)
    s = api.solve_grad("linear", P, Y, wl["t0"], wl["t1"], wl["save_t"], wl["rtol"], wl["atol"], layout="soa",
                       method="tsit5")
    rec, _, _ = api.forward_record("linear", P, Y, wl["t0"], wl["t1"], wl["save_t"], wl["rtol"], wl["atol"],
                                   layout="soa", want_saves=False, method="tsit5")
    g = api.reverse(rec, P, Y, layout="soa")
    np.testing.assert_array_equal(s["params_bar"].cpu().numpy(), g["params_bar"].cpu().numpy())
