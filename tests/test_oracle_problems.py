"""Pins of the right-hand sides and of their dual-number Jacobians.

Properties fixed by the mathematics of each model (paper Appendix A), not by
re-typing its formula: equilibria of Lorenz, conservation in Robertson and
HIRES, the trace and determinant of Van der Pol's linearisation at the origin,
and the zero-network limit of the LV UDE. The dual-number Jacobian is checked
against central differences of f.
"""
import numpy as np
import pytest

import oracle
from paper_2609_02876_gb300 import workloads as W


@pytest.mark.parametrize("name", ["lorenz", "vdp", "robertson", "hires", "linear", "lv_ude"])
def test_jacobian_matches_central_differences(name):
    d, P, _, nw = oracle.problem_info(name)
    rng = np.random.default_rng(1)
    y = rng.uniform(0.2, 1.5, (5, d))
    if name == "hires":
        p = np.tile(W.HIRES_RATES, (5, 1))
    elif name == "robertson":
        p = np.tile(W.ROBERTSON_RATES, (5, 1))
    else:
        p = rng.uniform(0.5, 2.0, (5, P))
    w = W.glorot_mlp(0) if nw else None
    f, J = oracle.rhs(name, p, y, w=w)
    for a in range(d):
        eps = 1e-6 * np.maximum(1.0, np.abs(y[:, a]))
        yp, ym = y.copy(), y.copy()
        yp[:, a] += eps
        ym[:, a] -= eps
        fd = (oracle.rhs(name, p, yp, w=w)[0] - oracle.rhs(name, p, ym, w=w)[0]) / (2 * eps[:, None])
        np.testing.assert_allclose(J[:, :, a], fd, rtol=1e-6, atol=1e-6 * np.abs(J).max())


def test_lorenz_equilibria():
    sig, rho, beta = 10.0, 28.0, 8.0 / 3.0
    r = np.sqrt(beta * (rho - 1.0))
    pts = np.array([[0.0, 0.0, 0.0], [r, r, rho - 1.0], [-r, -r, rho - 1.0]])
    f, _ = oracle.rhs("lorenz", np.tile([sig, rho, beta], (3, 1)), pts)
    assert np.abs(f).max() < 1e-12


def test_vdp_linearisation_at_origin():
    for mu in (0.5, 1.0, 2.0):
        f, J = oracle.rhs("vdp", [[mu]], [[0.0, 0.0]])
        assert np.abs(f).max() == 0.0
        assert np.isclose(np.trace(J[0]), mu) and np.isclose(np.linalg.det(J[0]), mu)


def test_conservation_of_rhs():
    rng = np.random.default_rng(2)
    y = rng.uniform(0, 1, (8, 3))
    f, _ = oracle.rhs("robertson", np.tile(W.ROBERTSON_RATES, (8, 1)), y)
    assert np.abs(f.sum(1)).max() < 1e-9 * 3e7
    y = rng.uniform(0, 1, (8, 8))
    f, _ = oracle.rhs("hires", np.tile(W.HIRES_RATES, (8, 1)), y)
    assert np.abs(f[:, 6] + f[:, 7]).max() < 1e-12


def test_lv_ude_zero_network_is_exponential():
    # With all weights zero the network outputs 0: x = x0 e^{a t}, y = y0 e^{-d t}.
    w = np.zeros(W.UDE_NW)
    p = np.array([[1.2, 2.5]])
    y0 = np.array([[0.8, 1.3]])
    rec = oracle.record("lv_ude", p, y0, 0.0, 5.0, [2.0, 5.0], 1e-10, 1e-12, w=w)
    exact = np.array([[0.8 * np.exp(1.2 * t), 1.3 * np.exp(-2.5 * t)] for t in (2.0, 5.0)])
    np.testing.assert_allclose(rec["y_save"][0], exact, rtol=1e-7)
