"""Pins of the oracle's record map R (adaptive solve, paper Sec. 2.1 and 3.1).

The step-size controller and starting step are readings of a paper that names
them without constants (an integral controller; the controller picks the first
step). They are pinned by what the paper prints about their result: the
accepted-step statistics of the Lorenz timing ensemble (Table 'dispersion'),
and accuracy against an independent high-accuracy solve (scipy DOP853 / Radau
at tight tolerance, the matching rule of Appendix B.1).
"""
import json
import os

import numpy as np
import pytest
from scipy.integrate import solve_ivp

import oracle
from paper_2609_02876_gb300 import workloads as W

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def test_lorenz_step_count_dispersion_matches_paper():
    g = GOLDEN["lorenz_dispersion"]
    wl = W.make("lorenz_paper", 1024)
    rec = oracle.record(wl["problem"], wl["params"], wl["y0"], wl["t0"], wl["t1"], wl["save_t"], wl["rtol"],
                        wl["atol"])
    mean, mx = rec["S"].mean(), rec["S"].max()
    # the paper's two step counters (its fused recorder and torchode) bracket 36.7..39 / 49..52;
    # the controller constants are not printed, so allow 10% around that bracket
    assert 0.9 * g["fused_recorder"]["mean"] <= mean <= 1.1 * g["torchode_counters"]["mean"]
    assert 0.9 * g["fused_recorder"]["max"] <= mx <= 1.1 * g["torchode_counters"]["max"]
    assert abs(mx / mean - g["fused_recorder"]["max_over_mean"]) < 0.1


def test_problem_constants_match_paper():
    np.testing.assert_array_equal(W.HIRES_RATES, GOLDEN["hires"]["literal_constants_in_order_of_first_appearance"])
    np.testing.assert_array_equal(W.HIRES_Y0, GOLDEN["hires"]["y0"])
    np.testing.assert_array_equal(W.ROBERTSON_RATES, GOLDEN["robertson"]["rates_k1_k2_k3"])
    # the oracle's HIRES right-hand side with the paper's constants conserves y7 + y8 and
    # is stationary in y7 + y8 only; a wrong constant assignment would break the pins in
    # test_oracle_invariants / test_oracle_problems


def _scipy_rhs(name, p):
    if name == "lorenz":
        return lambda t, y: [p[0] * (y[1] - y[0]), y[0] * (p[1] - y[2]) - y[1], y[0] * y[1] - p[2] * y[2]]
    if name == "vdp":
        return lambda t, y: [y[1], p[0] * ((1 - y[0] ** 2) * y[1] - y[0])]
    if name == "robertson":
        return lambda t, y: [-p[0] * y[0] + p[2] * y[1] * y[2],
                             p[0] * y[0] - p[2] * y[1] * y[2] - p[1] * y[1] ** 2, p[1] * y[1] ** 2]
    if name == "hires":
        def f(t, y):
            return [-p[0] * y[0] + p[1] * y[1] + p[2] * y[2] + p[3], p[0] * y[0] - p[4] * y[1],
                    -p[5] * y[2] + p[1] * y[3] + p[6] * y[4], p[2] * y[1] + p[0] * y[2] - p[7] * y[3],
                    -p[8] * y[4] + p[1] * y[5] + p[1] * y[6],
                    -p[9] * y[5] * y[7] + p[10] * y[3] + p[0] * y[4] - p[1] * y[5] + p[10] * y[6],
                    p[9] * y[5] * y[7] - p[11] * y[6], -p[9] * y[5] * y[7] + p[11] * y[6]]
        return f
    raise KeyError(name)


@pytest.mark.parametrize("name,method,med_bound,max_bound", [
    ("lorenz", "DOP853", 5e-6, 1e-4),
    ("vdp", "DOP853", 5e-5, 1e-3),
    ("robertson", "Radau", 1e-4, 1e-3),
    ("hires", "Radau", 1e-4, 1e-2),
])
def test_record_accuracy_against_independent_solver(name, method, med_bound, max_bound):
    """Matched-error metric of Appendix B.1: median (and max) over all save-time
    components of |y - y_ref| / max(|y_ref|, 1e-30), with y_ref from scipy."""
    n = 4
    wl = W.make(name, n)
    rec = oracle.record(wl["problem"], wl["params"], wl["y0"], wl["t0"], wl["t1"], wl["save_t"], wl["rtol"],
                        wl["atol"])
    assert (rec["status"] == 0).all()
    errs = []
    for k in range(n):
        sol = solve_ivp(_scipy_rhs(name, wl["params"][k]), (wl["t0"], wl["t1"]), wl["y0"][k], method=method,
                        t_eval=wl["save_t"], rtol=1e-12 if method == "DOP853" else 1e-10,
                        atol=1e-14 if method == "DOP853" else 1e-14)
        assert sol.success
        ref = sol.y.T
        big = np.abs(ref) > 1e3 * wl["atol"]  # components resolved above the absolute tolerance
        errs.append((np.abs(rec["y_save"][k] - ref) / np.maximum(np.abs(ref), 1e-30))[big])
    e = np.concatenate(errs)
    assert np.median(e) < med_bound, np.median(e)
    assert e.max() < max_bound, e.max()


@pytest.mark.parametrize("name,rtol,med_bound,max_bound", [("lorenz", 1e-6, 1e-7, 5e-6), ("vdp", 1e-8, 2e-9, 2e-6)])
def test_verner7_record_accuracy_against_independent_solver(name, rtol, med_bound, max_bound):
    """The seventh-order pair's adaptive solve against scipy's DOP853 at rtol 1e-13.
    The bounds sit below what Tsit5 reaches at the same tolerance (Lorenz,
    rtol 1e-6: median 3.7e-7, max 3.6e-5; Van der Pol, rtol 1e-8: 3.5e-9,
    2.4e-6) and above Verner7's (1.6e-8, 4.9e-7; 5.9e-10, 4.3e-7)."""
    n = 4
    wl = W.make(name, n, rtol=rtol)
    rec = oracle.record(wl["problem"], wl["params"], wl["y0"], wl["t0"], wl["t1"], wl["save_t"], wl["rtol"],
                        wl["atol"], method=oracle.METHOD_VERNER7)
    assert (rec["status"] == 0).all()
    errs = []
    for k in range(n):
        sol = solve_ivp(_scipy_rhs(name, wl["params"][k]), (wl["t0"], wl["t1"]), wl["y0"][k], method="DOP853",
                        t_eval=wl["save_t"], rtol=1e-13, atol=1e-15)
        assert sol.success
        ref = sol.y.T
        big = np.abs(ref) > 1e3 * wl["atol"]
        errs.append((np.abs(rec["y_save"][k] - ref) / np.maximum(np.abs(ref), 1e-30))[big])
    e = np.concatenate(errs)
    assert np.median(e) < med_bound, np.median(e)
    assert e.max() < max_bound, e.max()


def test_mesh_is_consistent():
    wl = W.make("vdp", 8)
    rec = oracle.record(wl["problem"], wl["params"], wl["y0"], wl["t0"], wl["t1"], wl["save_t"], wl["rtol"],
                        wl["atol"])
    for k in range(8):
        h = rec["h"][rec["offsets"][k]:rec["offsets"][k + 1]]
        assert (h > 0).all()
        assert abs(h.sum() - (wl["t1"] - wl["t0"])) < 1e-12 * wl["t1"]
        assert rec["n_att"][k] >= rec["S"][k]


def test_status_codes():
    wl = W.make("lorenz", 4)
    p = wl["params"].copy()
    p[1, 0] = np.nan
    rec = oracle.record(wl["problem"], p, wl["y0"], wl["t0"], wl["t1"], wl["save_t"], wl["rtol"], wl["atol"])
    assert rec["status"].tolist() == [oracle.TRAJ_OK, oracle.TRAJ_NONFINITE, oracle.TRAJ_OK, oracle.TRAJ_OK]
    rec = oracle.record(wl["problem"], wl["params"], wl["y0"], wl["t0"], wl["t1"], wl["save_t"], wl["rtol"],
                        wl["atol"], max_steps=5)
    assert (rec["status"] == oracle.TRAJ_MAXSTEPS).all()
    assert (rec["n_att"] == 5).all()


def test_gradient_accuracy_against_an_independent_sensitivity():
    """The replay gradient is an accurate sensitivity of the ODE, not only a
    self-consistent derivative: on the paper's Lorenz ensemble (rho over [0, 21],
    rtol 1e-6, atol 1e-9, loss ||y(t1)||^2) it agrees with central differences of a
    separately and tightly solved reference at the level of the forward error, as
    the paper's gradient-accuracy table reports (4.6e-6 for Lorenz). The
    median relative difference here must sit at that level, within 2 decades."""
    n = 64
    wl = W.make("lorenz_paper", n)
    P, Y0 = wl["params"], wl["y0"]
    g = oracle.solve_grad("lorenz", P, Y0, 0.0, 1.0, [1.0], 1e-6, 1e-9)

    def loss(p):
        r = oracle.record("lorenz", p, Y0, 0.0, 1.0, [1.0], 1e-12, 1e-14)
        return (r["y_save"][:, 0, :] ** 2).sum(1)

    ref = np.zeros_like(P)
    for q in range(3):
        e = np.zeros_like(P)
        e[:, q] = 1e-5 * np.maximum(np.abs(P[:, q]), 1e-3)
        ref[:, q] = (loss(P + e) - loss(P - e)) / (2 * e[:, q])
    rel = np.abs(g["params_bar"] - ref).max(1) / np.abs(ref).max(1)
    fwd = oracle.record("lorenz", P, Y0, 0.0, 1.0, [1.0], 1e-6, 1e-9)["y_save"][:, 0, :]
    tight = oracle.record("lorenz", P, Y0, 0.0, 1.0, [1.0], 1e-12, 1e-14)["y_save"][:, 0, :]
    ferr = np.abs(fwd - tight).max(1) / np.abs(tight).max(1)
    assert 4.6e-8 < np.median(rel) < 4.6e-4, np.median(rel)
    assert np.median(rel) < 30 * np.median(ferr) + 1e-12, (np.median(rel), np.median(ferr))


def test_hires_rodas5p_gradient_accuracy_is_the_papers_order():
    """Sec. 5 reports the Rodas5P replay reaching an achieved error of 1.3e-7 on
    HIRES (tolerance not stated). At rtol 1e-6, atol 1e-10 the oracle's gradient
    with respect to y0 sits at or below that level against a converged solve
    (rtol 1e-11), and is not exact (a loose check on the Rodas5P table and the
    step control together)."""
    wl = W.make("hires", 4)

    def grad(rtol, atol):
        return oracle.solve_grad("hires", wl["params"], wl["y0"], wl["t0"], wl["t1"], wl["save_t"], rtol, atol,
                                 method=oracle.METHOD_RODAS5P)

    g, ref = grad(1e-6, 1e-10), grad(1e-11, 1e-15)
    e = np.abs(g["y0_bar"] - ref["y0_bar"]).max(1) / np.abs(ref["y0_bar"]).max(1)
    assert e.max() < 2 * 1.3e-7 and e.min() > 1e-11, e
