"""Pins of the oracle's Rosenbrock23 (Shampine & Reichelt 1997; the paper's
second-order stiff method, Sec. 3.2) against facts that do not come from its
own formulas:

- its stability function R(z) (one step of y' = lambda y) agrees with e^z to
  second order, vanishes at z -> -infinity (L-stability) and keeps |R| <= 1 on
  the imaginary axis (a rotation is never amplified);
- its error estimate is the step's true local error to leading order, and
  y_new + e is third order;
- on a nonlinear problem the replay converges with order 2;
- it conserves Robertson's total mass (a linear invariant of f);
- its discrete adjoint equals a dual-number JVP of the same replay and central
  finite differences (as for the other methods).
"""
import numpy as np
import pytest

import oracle
from paper_2609_02876_gb300 import workloads as W

R23 = oracle.METHOD_ROSENBROCK23


def one_step(A, y0, h):
    """One Rosenbrock23 step of y' = A y (2x2, row-major params) for each h."""
    h = np.atleast_1d(np.asarray(h, dtype=np.float64))
    p = np.tile(np.asarray(A, dtype=np.float64).reshape(1, 4), (h.size, 1))
    y = np.tile(np.asarray(y0, dtype=np.float64).reshape(1, 2), (h.size, 1))
    return oracle.step("linear", R23, p, y, h)


def test_stability_function_is_second_order():
    lam = -1.3
    hs = np.array([0.04, 0.02, 0.01, 0.005])
    yn, _ = one_step([lam, 0, 0, 0], [1.0, 0.0], hs)
    err = np.abs(yn[:, 0] - np.exp(lam * hs))
    ratios = err[:-1] / err[1:]
    assert np.all((ratios > 7.0) & (ratios < 9.0)), ratios  # local error O(z^3)


def test_l_stability_and_imaginary_axis():
    yn, _ = one_step([-1.0, 0, 0, 0], [1.0, 0.0], [1e4, 1e6, 1e8])
    assert np.all(np.abs(yn[:, 0]) < 1e-3) and abs(yn[-1, 0]) < 1e-7
    w = 1.0
    yn, _ = one_step([0.0, w, -w, 0.0], [1.0, 0.5], np.logspace(-3, 4, 29))
    assert np.all(np.linalg.norm(yn, axis=1) <= np.linalg.norm([1.0, 0.5]) * (1 + 1e-14))


def test_error_estimate_is_the_local_error_to_leading_order():
    """e = (third-order solution) - y_new, so e / (y_new - exact) -> -1 as h -> 0."""
    lam = 0.7
    for h in (0.02, 0.01):
        yn, e = one_step([lam, 0, 0, -2.0], [1.0, 1.0], h)
        true = yn[0] - np.exp(np.array([lam, -2.0]) * h)
        np.testing.assert_allclose(e[0] / true, -1.0, atol=0.01 * h / 0.01)


def test_embedded_solution_is_third_order():
    """y_new + e is the pair's third-order solution: its local error falls by 16
    per halving of h (against 8 for y_new); a wrong e32 leaves it at 8."""
    for lam in (-1.3, 0.7):
        hs = np.array([0.08, 0.04, 0.02, 0.01])
        yn, e = one_step([lam, 0, 0, 0], [1.0, 0.0], hs)
        err3 = np.abs(yn[:, 0] + e[:, 0] - np.exp(lam * hs))
        r = err3[:-1] / err3[1:]
        assert np.all((r > 14.5) & (r < 18.0)), r


def test_replay_converges_with_order_two():
    wl = W.make("vdp", 1)
    p, y0 = np.array([[1.0]]), np.array([[1.5, -0.5]])
    ref = oracle.record("vdp", p, y0, 0.0, 2.0, [2.0], 1e-12, 1e-14)["y_save"][0, 0]
    errs = []
    for N in (200, 400, 800):
        h = np.full(N, 2.0 / N)
        o = oracle.replay_grad("vdp", p, y0, 0.0, 2.0, [2.0], np.array([0, N]), h, method=R23)
        errs.append(np.abs(o["y_save"][0, 0] - ref).max())
    r = np.array(errs[:-1]) / np.array(errs[1:])
    assert np.all((r > 3.6) & (r < 4.4)), r
    del wl


def test_record_conserves_robertson_mass():
    wl = W.make("robertson", 6)
    rec = oracle.record("robertson", wl["params"], wl["y0"], wl["t0"], wl["t1"], wl["save_t"], wl["rtol"], wl["atol"],
                        method=R23)
    assert (rec["status"] == 0).all()
    np.testing.assert_allclose(rec["y_save"].sum(2), 1.0, atol=1e-12)
    assert (rec["S"] > 20).all()


def _setup(name, n):
    if name == "linear":
        rng = np.random.default_rng(4)
        A = np.array([[-50.0, 1.0, 2.0, -3.0]]) * (1 + 0.1 * rng.standard_normal((n, 4)))
        wl = dict(problem="linear", params=A, y0=rng.standard_normal((n, 2)), t0=0.0, t1=1.0,
                  save_t=np.linspace(0.1, 1.0, 10), rtol=1e-6, atol=1e-9, w=None)
    else:
        wl = W.make(name, n)
    rec = oracle.record(wl["problem"], wl["params"], wl["y0"], wl["t0"], wl["t1"], wl["save_t"], wl["rtol"],
                        wl["atol"], method=R23)
    assert (rec["status"] == 0).all()
    return wl, rec


def _grad(wl, rec, params=None, y0=None, ybar=None):
    return oracle.replay_grad(wl["problem"], wl["params"] if params is None else params,
                              wl["y0"] if y0 is None else y0, wl["t0"], wl["t1"], wl["save_t"], rec["offsets"],
                              rec["h"], ybar_save=ybar, method=R23)


@pytest.mark.parametrize("name", ["robertson", "hires", "linear"])
def test_adjoint_equals_dual_number_jvp(name):
    wl, rec = _setup(name, 4)
    n, P = wl["params"].shape
    d = wl["y0"].shape[1]
    rng = np.random.default_rng(13)
    pdot = rng.standard_normal((n, P)) * wl["params"]
    ydot = rng.standard_normal((n, d))
    g = _grad(wl, rec)
    j = oracle.replay_jvp(wl["problem"], wl["params"], wl["y0"], wl["t0"], wl["t1"], wl["save_t"], rec["offsets"],
                          rec["h"], pdot, ydot, method=R23)
    np.testing.assert_allclose(j["loss"], g["loss"], rtol=1e-15)
    lhs = (g["params_bar"] * pdot).sum(1) + (g["y0_bar"] * ydot).sum(1)
    scale = np.abs(g["params_bar"] * pdot).sum(1) + np.abs(g["y0_bar"] * ydot).sum(1)
    assert np.all(np.abs(lhs - j["loss_dot"]) <= 1e-12 * scale)
    ybar = rng.standard_normal(g["y_save"].shape)
    gu = _grad(wl, rec, ybar=ybar)
    lhs = (gu["params_bar"] * pdot).sum(1) + (gu["y0_bar"] * ydot).sum(1)
    rhs = (ybar * j["y_save_dot"]).sum((1, 2))
    scale = np.abs(gu["params_bar"] * pdot).sum(1) + np.abs(gu["y0_bar"] * ydot).sum(1)
    assert np.all(np.abs(lhs - rhs) <= 1e-12 * scale)


@pytest.mark.parametrize("name", ["robertson", "hires", "linear"])
def test_adjoint_matches_central_fd_on_same_mesh(name):
    wl, rec = _setup(name, 3)
    n, P = wl["params"].shape
    g = _grad(wl, rec)
    rng = np.random.default_rng(1)
    v = rng.standard_normal((n, P + wl["y0"].shape[1]))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    x = np.concatenate([wl["params"], wl["y0"]], 1)
    dx = v * 1e-6 * np.maximum(np.abs(x), 1e-3)
    lp = _grad(wl, rec, params=(x + dx)[:, :P], y0=(x + dx)[:, P:])["loss"]
    lm = _grad(wl, rec, params=(x - dx)[:, :P], y0=(x - dx)[:, P:])["loss"]
    fd = (lp - lm) / 2.0
    ad = (np.concatenate([g["params_bar"], g["y0_bar"]], 1) * dx).sum(1)
    assert (np.abs(fd - ad) / np.abs(ad)).max() < 1e-5


@pytest.mark.parametrize("name,med_bound,max_bound", [("robertson", 2e-6, 1e-2), ("hires", 2e-7, 1e-4)])
def test_record_accuracy_against_radau(name, med_bound, max_bound):
    """The adaptive Rosenbrock23 solve at the workload's tolerance against scipy's
    Radau at rtol 1e-10: the save states match to the accuracy a second-order
    method reaches there (Robertson median 2.9e-7, HIRES 3.0e-8 measured)."""
    from scipy.integrate import solve_ivp
    from tests.test_oracle_record import _scipy_rhs
    wl = W.make(name, 4)
    rec = oracle.record(wl["problem"], wl["params"], wl["y0"], wl["t0"], wl["t1"], wl["save_t"], wl["rtol"],
                        wl["atol"], method=R23)
    assert (rec["status"] == 0).all()
    errs = []
    for k in range(4):
        sol = solve_ivp(_scipy_rhs(name, wl["params"][k]), (wl["t0"], wl["t1"]), wl["y0"][k], method="Radau",
                        t_eval=wl["save_t"], rtol=1e-10, atol=1e-14)
        assert sol.success
        big = np.abs(sol.y.T) > 1e3 * wl["atol"]
        errs.append((np.abs(rec["y_save"][k] - sol.y.T) / np.abs(sol.y.T))[big])
    e = np.concatenate(errs)
    assert np.median(e) < med_bound and e.max() < max_bound, (np.median(e), e.max())
