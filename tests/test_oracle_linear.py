"""Closed-form pins of the oracle's replay and discrete adjoint on dy/dt = A(theta) y.

For a linear right-hand side one Tsit5 step is exactly y_new = R(hA) y with the
stability polynomial R(z) = 1 + sum_q (b^T A_rk^{q-1} 1) z^q, and one Rodas5P step
with the exact Jacobian J = A is exactly y_new = (I + sum_i b_i K_i) y with
K_i = (I - gamma hA)^{-1} hA (I + sum_{j<i} (alpha_ij + gamma_ij) K_j).
The replay (paper Eq. (replay)) is therefore a matrix product, and its gradient
follows by complex-step differentiation of that product (exact to roundoff,
no finite-difference error). Neither uses the oracle's stage or adjoint code.
"""
import numpy as np
import pytest
from scipy.linalg import expm, expm_frechet

import oracle
from tests.test_oracle_tableau import rodas_standard


def _mesh_times(t0, t1, h):
    ts = [t0]
    for i, hi in enumerate(h):
        ts.append(t1 if i == len(h) - 1 else ts[-1] + hi)
    return np.array(ts)


def _tsit5_R(tab):
    """Stability polynomial of an explicit tableau (Tsit5, Verner7)."""
    A, b = tab["A"], tab["b"]
    s = A.shape[0]
    beta = [b @ np.linalg.matrix_power(A, q - 1) @ np.ones(s) for q in range(1, s + 1)]

    def R(Z):
        out = np.eye(Z.shape[0], dtype=Z.dtype)
        Zq = np.eye(Z.shape[0], dtype=Z.dtype)
        for q in range(1, s + 1):
            Zq = Zq @ Z
            out = out + beta[q - 1] * Zq
        return out

    return R


def _rodas_R(tab):
    alpha, G, b = rodas_standard(tab)
    gam = tab["gamma"]
    Bs = np.tril(alpha + G, -1)

    def R(Z):
        d = Z.shape[0]
        I = np.eye(d, dtype=Z.dtype)
        M = np.linalg.inv(I - gam * Z)
        K = []
        for i in range(8):
            acc = I.copy()
            for j in range(i):
                acc = acc + Bs[i, j] * K[j]
            K.append(M @ Z @ acc)
        out = I.copy()
        for i in range(8):
            out = out + b[i] * K[i]
        return out

    return R


def closed_form_loss(R, theta, y0, t0, t1, h, save_t):
    A = np.array([[theta[0], theta[1]], [theta[2], theta[3]]])
    ts = _mesh_times(t0, t1, h)
    ys = [y0]
    for hi in h:
        ys.append(R(hi * A) @ ys[-1])
    L = 0.0
    out = []
    for s in save_t:
        i = max(i for i in range(len(ts)) if ts[i] <= s)
        hs = s - ts[i]
        ysv = ys[i] if hs == 0.0 else R(hs * A) @ ys[i]
        out.append(ysv)
        L = L + np.sum(ysv * ysv)
    return L, np.array(out)


def complex_step_grad(R, theta, y0, t0, t1, h, save_t, eps=1e-30):
    gth = np.zeros(4)
    gy = np.zeros(2)
    for p in range(4):
        th = theta.astype(complex)
        th[p] += 1j * eps
        gth[p] = closed_form_loss(R, th, y0.astype(complex), t0, t1, h, save_t)[0].imag / eps
    for c in range(2):
        y = y0.astype(complex)
        y[c] += 1j * eps
        gy[c] = closed_form_loss(R, theta.astype(complex), y, t0, t1, h, save_t)[0].imag / eps
    return gth, gy


CASES = [
    # (method, theta, step sizes): mild, oscillatory, stiff (Rodas only)
    (oracle.METHOD_TSIT5, [-0.3, 0.8, -0.9, 0.1], 0.07),
    (oracle.METHOD_TSIT5, [0.2, 1.5, -1.5, -0.1], 0.15),
    (oracle.METHOD_RODAS5P, [-0.3, 0.8, -0.9, 0.1], 0.07),
    (oracle.METHOD_RODAS5P, [-1000.0, 1.0, 0.5, -1.0], 0.4),
    (oracle.METHOD_VERNER7, [-0.3, 0.8, -0.9, 0.1], 0.07),
    (oracle.METHOD_VERNER7, [0.2, 1.5, -1.5, -0.1], 0.3),
]


@pytest.mark.parametrize("method,theta,hscale", CASES)
def test_replay_and_adjoint_match_closed_form(method, theta, hscale):
    rng = np.random.default_rng(7)
    theta = np.array(theta)
    y0 = np.array([0.7, -0.4])
    h = hscale * rng.uniform(0.5, 1.5, 23)
    t0 = 0.25
    t1 = t0
    for hi in h[:-1]:
        t1 = t1 + hi
    t1 = t1 + h[-1]
    ts = _mesh_times(t0, t1, h)
    # save times: interior points, one exactly on a mesh point, and t1 itself
    save_t = np.sort(np.concatenate([rng.uniform(t0 + 1e-3, t1 - 1e-3, 6), [ts[9], t1]]))
    tab = oracle.tableau(method)
    R = _rodas_R(tab) if method == oracle.METHOD_RODAS5P else _tsit5_R(tab)
    L_ref, ysv_ref = closed_form_loss(R, theta, y0, t0, t1, h, save_t)
    gth_ref, gy_ref = complex_step_grad(R, theta, y0, t0, t1, h, save_t)
    off = np.array([0, len(h)])
    g = oracle.replay_grad("linear", theta[None], y0[None], t0, t1, save_t, off, h, method=method)
    assert g["ok"].all()
    np.testing.assert_allclose(g["y_save"][0], ysv_ref, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(g["loss"][0], L_ref, rtol=1e-13)
    scale = np.abs(gth_ref).max()
    np.testing.assert_allclose(g["params_bar"][0], gth_ref, rtol=1e-11, atol=1e-12 * scale)
    np.testing.assert_allclose(g["y0_bar"][0], gy_ref, rtol=1e-11, atol=1e-12 * np.abs(gy_ref).max())


@pytest.mark.parametrize("method", [oracle.METHOD_TSIT5, oracle.METHOD_RODAS5P])
def test_linear_family_accuracy_and_sensitivity(method):
    """The paper's linear family dy_i/dt = 1.01 y_i on [0, 10] (Appendix A): the
    solution y0 e^{10.1}; and a non-normal A whose exact sensitivity comes from
    the Frechet derivative of expm. The replay's gradient matches the exact
    sensitivity to the method's forward error (paper Appendix B.6)."""
    n = 16
    rng = np.random.default_rng(3)
    y0 = rng.uniform(0.1, 1.0, (n, 2))
    theta = np.tile([1.01, 0.0, 0.0, 1.01], (n, 1))
    rtol = 1e-8
    rec = oracle.record("linear", theta, y0, 0.0, 10.0, [10.0], rtol, 1e-14, method=method)
    assert (rec["status"] == 0).all()
    # every trajectory takes the same steps (paper Table dispersion: equal counts)
    assert len(set(rec["S"].tolist())) == 1
    exact = y0 * np.exp(10.1)
    rel = np.abs(rec["y_save"][:, 0, :] - exact) / exact
    assert rel.max() < 2e-5

    th = np.array([-0.4, 1.2, -0.7, -0.2])
    T = 3.0
    yy = np.array([0.3, 0.9])
    rec = oracle.record("linear", th[None], yy[None], 0.0, T, [T], rtol, 1e-12, method=method)
    g = oracle.replay_grad("linear", th[None], yy[None], 0.0, T, [T], rec["offsets"], rec["h"], method=method)
    A = th.reshape(2, 2)
    yT = expm(T * A) @ yy
    gy_exact = 2.0 * expm(T * A).T @ yT
    gth_exact = np.zeros(4)
    for p in range(4):
        E = np.zeros(4)
        E[p] = 1.0
        _, dM = expm_frechet(T * A, T * E.reshape(2, 2))
        gth_exact[p] = 2.0 * yT @ (dM @ yy)
    np.testing.assert_allclose(g["y_save"][0, 0], yT, rtol=1e-6)
    np.testing.assert_allclose(g["params_bar"][0], gth_exact, rtol=1e-5, atol=1e-6)
    np.testing.assert_allclose(g["y0_bar"][0], gy_exact, rtol=1e-5)


def test_planted_adjoint_sign_error_is_detected():
    # A wrong sign in one stage weight changes the closed-form gradient visibly.
    tab = oracle.tableau(oracle.METHOD_TSIT5)
    tab_bad = {k: (v.copy() if hasattr(v, "copy") else v) for k, v in tab.items()}
    tab_bad["b"][3] = -tab_bad["b"][3]
    theta = np.array([-0.3, 0.8, -0.9, 0.1])
    y0 = np.array([0.7, -0.4])
    h = np.full(10, 0.1)
    g_good = complex_step_grad(_tsit5_R(tab), theta, y0, 0.0, 1.0, h, [1.0])[0]
    g_bad = complex_step_grad(_tsit5_R(tab_bad), theta, y0, 0.0, 1.0, h, [1.0])[0]
    assert np.abs(g_good - g_bad).max() > 1e-3 * np.abs(g_good).max()
