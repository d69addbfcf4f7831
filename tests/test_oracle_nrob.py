"""Pins of the oracle's Robertson neural right-hand side (paper Appendix A):
Robertson with its k2 y2^2 term replaced by a shared MLP 3-16-16-1 (tanh,
softplus output) in both the sink and the source.

- the neural term moves mass between species 2 and 3 only, so the total mass
  stays 1 along the record;
- the shared-weight gradient of the stiff adjoint (first-order terms through
  the stage VJPs plus the weight derivative of the Jacobian contraction)
  equals central finite differences of the replay loss along random weight
  directions, for Rodas5P and Rosenbrock23;
- with the output layer zeroed the network is a constant, and no gradient
  reaches the hidden layers;
- the per-trajectory adjoint equals a dual-number JVP of the same replay.
"""
import numpy as np
import pytest

import oracle
from paper_2609_02876_gb300 import workloads as W

METHODS = [oracle.METHOD_RODAS5P, oracle.METHOD_ROSENBROCK23]


def _short(n, w=None):
    """A shorter span (t in [1e-5, 10]) keeps the finite differences quick."""
    wl = W.make("nrob", n)
    wl = dict(wl, t1=10.0, save_t=W.log_saves(1e-5, 10.0, 8))
    if w is not None:
        wl["w"] = w
    return wl


def _record(wl, method):
    rec = oracle.record("nrob", wl["params"], wl["y0"], wl["t0"], wl["t1"], wl["save_t"], wl["rtol"], wl["atol"],
                        method=method, w=wl["w"])
    assert (rec["status"] == 0).all()
    return rec


def _grad(wl, rec, method, w=None, params=None, y0=None):
    return oracle.replay_grad("nrob", wl["params"] if params is None else params, wl["y0"] if y0 is None else y0,
                              wl["t0"], wl["t1"], wl["save_t"], rec["offsets"], rec["h"], method=method,
                              w=wl["w"] if w is None else w)


def test_mass_is_conserved():
    wl = W.make("nrob", 3)
    rec = _record(wl, oracle.METHOD_RODAS5P)
    np.testing.assert_allclose(rec["y_save"].sum(2), 1.0, atol=1e-12)
    assert (rec["S"] > 50).all()


@pytest.mark.parametrize("method", METHODS)
def test_weight_gradient_matches_central_fd(method):
    wl = _short(2)
    rec = _record(wl, method)
    g = _grad(wl, rec, method)
    rng = np.random.default_rng(21)
    for _ in range(3):
        dw = rng.standard_normal(W.NROB_NW) * np.maximum(np.abs(wl["w"]), 1e-2) * 1e-6
        lp = _grad(wl, rec, method, w=wl["w"] + dw)["loss"].sum()
        lm = _grad(wl, rec, method, w=wl["w"] - dw)["loss"].sum()
        fd = (lp - lm) / 2.0
        ad = float(g["w_bar"] @ dw)
        assert abs(fd - ad) <= 1e-5 * abs(ad), (fd, ad)


def test_constant_network_sends_no_gradient_to_hidden_layers():
    w = W.glorot_nrob(0)
    w[336:352] = 0.0  # W3 = 0: NN(y) = softplus(b3)
    wl = _short(2, w=w)
    rec = _record(wl, oracle.METHOD_RODAS5P)
    g = _grad(wl, rec, oracle.METHOD_RODAS5P)
    assert np.all(g["w_bar"][:336] == 0.0)
    assert g["w_bar"][352] != 0.0


@pytest.mark.parametrize("method", METHODS)
def test_adjoint_equals_dual_number_jvp(method):
    wl = _short(3)
    rec = _record(wl, method)
    rng = np.random.default_rng(5)
    pdot = rng.standard_normal((3, 2)) * wl["params"]
    ydot = rng.standard_normal((3, 3)) * 1e-3
    g = _grad(wl, rec, method)
    j = oracle.replay_jvp("nrob", wl["params"], wl["y0"], wl["t0"], wl["t1"], wl["save_t"], rec["offsets"],
                          rec["h"], pdot, ydot, method=method, w=wl["w"])
    lhs = (g["params_bar"] * pdot).sum(1) + (g["y0_bar"] * ydot).sum(1)
    scale = np.abs(g["params_bar"] * pdot).sum(1) + np.abs(g["y0_bar"] * ydot).sum(1)
    assert np.all(np.abs(lhs - j["loss_dot"]) <= 1e-12 * scale)


def test_weight_derivative_of_the_jacobian_contraction_matches_fd():
    """The stiff adjoint's term d/dw (r^T J(y, w) u) against central differences
    of r^T J u, with J from the dual-number Jacobian at perturbed weights. The
    weight-free part of J does not enter the derivative; k3 = 0 here keeps its
    large entries from adding rounding to the differences, and the k1 part is
    removed using plain Robertson with k2 = k3 = 0."""
    rng = np.random.default_rng(17)
    w = W.glorot_nrob(0)
    p = np.array([[0.05, 0.0]])
    for _ in range(4):
        y = np.array([0.9, 3e-5, 0.1]) * (1 + 0.1 * rng.standard_normal(3))
        r, u = rng.standard_normal(3), rng.standard_normal(3)
        g = oracle.w_contract("nrob", y, w, r, u)
        _, Jr = oracle.rhs("robertson", np.array([[0.05, 0.0, 0.0]]), y[None])

        def G(ww):
            _, J = oracle.rhs("nrob", p, y[None], w=ww)
            return r @ (J[0] - Jr[0]) @ u

        dw = rng.standard_normal(W.NROB_NW) * 1e-6
        fd = (G(w + dw) - G(w - dw)) / 2.0
        assert abs(fd - g @ dw) <= 1e-6 * np.abs(g * dw).sum(), (fd, g @ dw)
