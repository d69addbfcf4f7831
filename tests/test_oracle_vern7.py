"""Pins of the oracle's seventh-order Verner pair (paper Sec. 5, higher-order
engines) against facts that do not come from its own step code.

The paper cites Verner (2010) for it and prints no table; the oracle holds
Verner's efficient 7(6) pair, whose order conditions and quadrature weights are
tested in test_oracle_tableau.py. Here:

- one step of y' = A y equals the stability polynomial R(hA) built from the
  table's b^T A^(q-1) 1 (the closed-form replay is in test_oracle_linear.py),
  and R agrees with e^z through z^7 but not z^8;
- the step's local error is O(h^8) and its error estimate O(h^7);
- on a nonlinear problem the local error is of order 8, and the replay of a
  linear system converges with order 7;
- at a tight tolerance the adaptive solve takes fewer steps than Tsit5 for the
  same accuracy;
- its discrete adjoint equals a dual-number JVP of the same replay and central
  finite differences.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2609_02876_gb300 import workloads as W

V7 = oracle.METHOD_VERNER7


def one_step(A, y0, h):
    h = np.atleast_1d(np.asarray(h, dtype=np.float64))
    p = np.tile(np.asarray(A, dtype=np.float64).reshape(1, 4), (h.size, 1))
    y = np.tile(np.asarray(y0, dtype=np.float64).reshape(1, 2), (h.size, 1))
    return oracle.step("linear", V7, p, y, h)


def stability_coeffs():
    tab = oracle.tableau(V7)
    A, b = tab["A"], tab["b"]
    return [1.0] + [b @ np.linalg.matrix_power(A, q - 1) @ np.ones(10) for q in range(1, 11)]


def test_stability_polynomial_is_seventh_order():
    beta = stability_coeffs()
    for q in range(8):
        # absolute: powers of A (entries up to 187) carry ~3e-15 of rounding
        assert abs(beta[q] - 1.0 / math.factorial(q)) < 1e-14, q
    assert abs(beta[8] - 1.0 / math.factorial(8)) > 1e-8  # not eighth order
    assert beta[10] == 0.0  # nine stages feed y_new


def test_one_linear_step_is_the_stability_polynomial():
    beta = stability_coeffs()
    Am = np.array([[-0.4, 1.3], [-1.1, 0.2]])
    y0 = np.array([0.6, -0.8])
    for h in (0.05, 0.3, 0.9):
        Z = h * Am
        R = sum(beta[q] * np.linalg.matrix_power(Z, q) for q in range(11))
        yn, _ = one_step(Am, y0, h)
        np.testing.assert_allclose(yn[0], R @ y0, rtol=1e-14, atol=1e-15)


def test_local_error_and_estimate_orders():
    """Scalar y' = lam y with lam > 0 (for lam < 0 the z^8 and z^9 error terms
    have opposite signs and nearly cancel at moderate z): |y_new - e^(lam h)|
    falls as h^8 (x256 per halving, up to the z^9 term) and the estimate |e| as
    h^7 (x128); the windows exclude the neighbouring orders."""
    for lam, h0 in ((0.7, 0.8), (2.5, 0.2)):
        hs = h0 / 2.0 ** np.arange(3)
        yn, _ = one_step([lam, 0, 0, 0], [1.0, 0.0], hs)
        loc = np.abs(yn[:, 0] - np.exp(lam * hs))
        r_loc = loc[:-1] / loc[1:]
        assert np.all((r_loc > 230) & (r_loc < 330)), r_loc
        hs = h0 / 2.0 ** np.arange(4)  # smaller steps take e into the rounding level
        _, e = one_step([lam, 0, 0, 0], [1.0, 0.0], hs)
        r_est = np.abs(e[:-1, 0]) / np.abs(e[1:, 0])
        assert np.all((r_est > 115) & (r_est < 155)), r_est


def test_nonlinear_local_error_is_eighth_order():
    """One step on Van der Pol (mu = 1) against 512 substeps of the same span:
    the local error falls as h^8 (x256 per halving; measured 240 and 237), which
    needs the nonlinear order conditions in the step code, not only the linear
    ones the stability polynomial checks."""
    p, y0 = np.array([[1.0]]), np.array([[1.5, -0.5]])
    errs = []
    for h in (0.4, 0.2, 0.1):
        one, _ = oracle.step("vdp", V7, p, y0, [h])
        N = 512
        ref = oracle.replay_grad("vdp", p, y0, 0.0, h, [h], np.array([0, N]), np.full(N, h / N),
                                 method=V7)["y_save"][0, 0]
        errs.append(np.abs(one[0] - ref).max())
    r = np.array(errs[:-1]) / np.array(errs[1:])
    assert np.all((r > 190) & (r < 330)), r


def test_replay_converges_with_order_seven():
    """Global error of N uniform steps on y' = A y over [0, 8] (A = [[0.5, 0.3],
    [-0.3, -0.5]]) against expm: x128 per halving in the limit (measured 106 and
    119 from N = 8 to 32, approaching it from below)."""
    import scipy.linalg as sl
    p, y0, T = np.array([[0.5, 0.3, -0.3, -0.5]]), np.array([[1.0, 0.5]]), 8.0
    exact = sl.expm(T * p[0].reshape(2, 2)) @ y0[0]
    errs = []
    for N in (8, 16, 32):
        o = oracle.replay_grad("linear", p, y0, 0.0, T, [T], np.array([0, N]), np.full(N, T / N), method=V7)
        errs.append(np.abs(o["y_save"][0, 0] - exact).max())
    r = np.array(errs[:-1]) / np.array(errs[1:])
    assert np.all((r > 90) & (r < 170)), r


def test_fewer_steps_than_tsit5_at_tight_tolerance():
    wl = W.make("lorenz", 8)
    args = (wl["params"], wl["y0"], wl["t0"], wl["t1"], wl["save_t"], 1e-10, 1e-12)
    v = oracle.record("lorenz", *args, method=V7)
    t = oracle.record("lorenz", *args, method=oracle.METHOD_TSIT5)
    ref = oracle.record("lorenz", *args[:5], 1e-13, 1e-15, method=V7)
    assert (v["status"] == 0).all() and (t["status"] == 0).all()
    assert v["S"].sum() < 0.6 * t["S"].sum()
    err_v = np.abs(v["y_save"] - ref["y_save"]).max()
    assert err_v < 1e-7, err_v


def _setup(name, n):
    if name == "linear":
        rng = np.random.default_rng(4)
        A = np.array([[-0.5, 1.0, -2.0, -0.3]]) * (1 + 0.1 * rng.standard_normal((n, 4)))
        wl = dict(problem="linear", params=A, y0=rng.standard_normal((n, 2)), t0=0.0, t1=3.0,
                  save_t=np.linspace(0.3, 3.0, 10), rtol=1e-8, atol=1e-10, w=None)
    else:
        wl = W.make(name, n)
    rec = oracle.record(wl["problem"], wl["params"], wl["y0"], wl["t0"], wl["t1"], wl["save_t"], wl["rtol"],
                        wl["atol"], method=V7)
    assert (rec["status"] == 0).all()
    return wl, rec


def _grad(wl, rec, params=None, y0=None, ybar=None):
    return oracle.replay_grad(wl["problem"], wl["params"] if params is None else params,
                              wl["y0"] if y0 is None else y0, wl["t0"], wl["t1"], wl["save_t"], rec["offsets"],
                              rec["h"], ybar_save=ybar, method=V7)


@pytest.mark.parametrize("name", ["lorenz", "vdp", "linear"])
def test_adjoint_equals_dual_number_jvp(name):
    wl, rec = _setup(name, 4)
    n, P = wl["params"].shape
    d = wl["y0"].shape[1]
    rng = np.random.default_rng(13)
    pdot = rng.standard_normal((n, P)) * wl["params"]
    ydot = rng.standard_normal((n, d))
    g = _grad(wl, rec)
    j = oracle.replay_jvp(wl["problem"], wl["params"], wl["y0"], wl["t0"], wl["t1"], wl["save_t"], rec["offsets"],
                          rec["h"], pdot, ydot, method=V7)
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


@pytest.mark.parametrize("name", ["lorenz", "vdp"])
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
