"""Pins of the oracle's record map R (the adaptive loop of the paper's Sec. 2.1:
weighted RMS error norm, accept when it is at most one, an integral
controller, the controller's own starting step) against scipy, an
implementation that shares nothing with the oracle.

- The starting step equals scipy's `select_initial_step` (Hairer, Norsett &
  Wanner I, Sec. II.4: the same RMS norm and Euler probe) called with the
  method's order, to 1e-12 relative (the probe's difference f(y0 + h0 f0) - f0
  cancels, which raises the two codes' rounding differences to ~1e-14).
- The accepted mesh equals that of scipy's explicit Runge-Kutta driver
  (`RungeKutta._step_impl`: safety 0.9, factor clamped to [0.2, 10], exponent
  -1/(q+1) for an error estimate of order q, factor capped at 1 after a
  rejection, scale atol + rtol max(|y|, |y_new|)) run with the oracle's Tsit5
  table (itself pinned by the order conditions) and the same starting step:
  the same number of accepted and attempted steps and the same h to 1e-6
  relative. The two codes round the stage sums differently (~1e-16 of |K|);
  the error estimate cancels down to ~1e-9 of |K| on smooth stretches, so err
  differs by up to ~1e-7 and each controller factor by ~1e-8 (measured:
  7e-8 on Van der Pol), and the differences compound over ~200 steps to
  ~5e-8 in h. A changed control constant moves h by 1e-3 or more.

The same driver run with Verner's 7(6) table (ten stages, the tenth used only
by the sixth-order estimate; error_estimator_order 6, exponent -1/7, starting
step of order 7) pins the oracle's Verner7 record: same counts, h to 3e-5
(the seventh-order estimate cancels further, and Van der Pol's many rejected
trials compound the rounding differences to 4e-6; measured).

For the Rosenbrock methods scipy has no driver of their own, so its
RungeKutta driver runs with its one-step function swapped for the oracle's
Rosenbrock step (itself pinned by its stability function, order and error
estimate), error_estimator_order set to the published embedded order
(Rosenbrock23 2, Shampine & Reichelt; Rodas5P 4, Steinebach) and the
starting step of the solution's order: scipy's accept test, safety factor,
clamps, exponent and post-rejection cap then drive the mesh, which must equal
the oracle's record (same counts, h to 1e-5: the two codes round the error
norm differently and Robertson's stiff control loop compounds that to ~1e-6).

A plausible mistake in the oracle's control constants must fail these pins;
the last tests plant several, one at a time, in a copy of the oracle compiled
here, and check that each one is caught.
"""
import contextlib
import os
import subprocess
import tempfile

import numpy as np
import pytest
from scipy.integrate import solve_ivp
from scipy.integrate._ivp.common import select_initial_step
from scipy.integrate._ivp.rk import RungeKutta

import oracle
from paper_2609_02876_gb300 import workloads as W

TSIT5 = oracle.METHOD_TSIT5
VERN7 = oracle.METHOD_VERNER7
H0_RTOL = 1e-12
H_RTOL = 1e-6  # h agreement (see the module docstring)
H_RTOL_V7 = 3e-5
H_RTOL_ROS = 1e-5
ROS23, RODAS5P = oracle.METHOD_ROSENBROCK23, oracle.METHOD_RODAS5P


def _rhs(name, p):
    if name == "lorenz":
        return lambda t, y: np.array([p[0] * (y[1] - y[0]), y[0] * (p[1] - y[2]) - y[1], y[0] * y[1] - p[2] * y[2]])
    if name == "vdp":
        return lambda t, y: np.array([y[1], p[0] * ((1 - y[0] ** 2) * y[1] - y[0])])
    raise KeyError(name)


def _tsit5_driver(order_for_first_step):
    tab = oracle.tableau(TSIT5)

    class Tsit5Scipy(RungeKutta):
        """scipy's RK driver with the Tsit5 table: six stages before y_new, the
        seventh (FSAL) stage is f(y_new), which scipy appends as K[-1]."""
        C = tab["c"][:6]
        A = tab["A"][:6, :6]
        B = tab["b"][:6]
        E = tab["b"] - tab["bhat"]
        P = np.zeros((7, 1))
        order = 5
        error_estimator_order = 4
        n_stages = 6

        def __init__(self, fun, t0, y0, t_bound, **kw):
            super().__init__(fun, t0, y0, t_bound, **kw)
            self.h_abs = select_initial_step(self.fun, self.t, self.y, t_bound, np.inf, self.f, self.direction,
                                             order_for_first_step, self.rtol, self.atol)

    return Tsit5Scipy


def _vern7_driver():
    tab = oracle.tableau(VERN7)

    class Vern7Scipy(RungeKutta):
        """scipy's RK driver with Verner's 7(6) table: all ten stages are computed
        (b_10 = 0: the tenth enters only the estimate), then f(y_new) as K[-1],
        which is the next step's first stage (the pair is not FSAL)."""
        C = tab["c"]
        A = tab["A"]
        B = tab["b"]
        E = np.append(tab["b"] - tab["bhat"], 0.0)
        P = np.zeros((11, 1))
        order = 7
        error_estimator_order = 6
        n_stages = 10

        def __init__(self, fun, t0, y0, t_bound, **kw):
            super().__init__(fun, t0, y0, t_bound, **kw)
            self.h_abs = select_initial_step(self.fun, self.t, self.y, t_bound, np.inf, self.f, self.direction,
                                             7, self.rtol, self.atol)

    return Vern7Scipy


def _scipy_mesh(name, p, y0, t0, t1, rtol, atol, method=TSIT5):
    drv, per_att = (_tsit5_driver(5), 6) if method == TSIT5 else (_vern7_driver(), 10)
    sol = solve_ivp(_rhs(name, p), (t0, t1), np.array(y0, dtype=np.float64), method=drv, rtol=rtol, atol=atol)
    assert sol.status == 0
    # nfev: f(y0), the starting-step probe (twice: scipy's own and the one above),
    # then per attempted step the stages after the first and f(y_new)
    return np.diff(sol.t), (sol.nfev - 3) // per_att


def _cases(method=TSIT5):
    out = []
    sets = ((("lorenz", 1e-6), ("lorenz", 1e-4), ("vdp", 1e-6), ("vdp", 1e-3)) if method == TSIT5 else
            (("lorenz", 1e-6), ("lorenz", 1e-4), ("lorenz", 1e-3), ("vdp", 1e-6)))
    for name, rtol in sets:
        wl = W.make(name, 24, rtol=rtol, seed=3)
        out.append((name, wl))
    return out


def _compare_meshes(cases, method=TSIT5):
    """Per trajectory: (equal accepted count, equal attempted count, max rel h diff
    over all steps but the last). Also returns the number of rejected trials seen."""
    res, rejected = [], 0
    for name, wl in cases:
        rec = oracle.record(name, wl["params"], wl["y0"], wl["t0"], wl["t1"], [], wl["rtol"], wl["atol"],
                            method=method, want_saves=False)
        for k in range(wl["params"].shape[0]):
            h_o = rec["h"][rec["offsets"][k]:rec["offsets"][k + 1]]
            h_s, att_s = _scipy_mesh(name, wl["params"][k], wl["y0"][k], wl["t0"], wl["t1"], wl["rtol"],
                                     wl["atol"], method)
            rejected += int(rec["n_att"][k] - rec["S"][k])
            if h_o.size != h_s.size:
                res.append((False, False, np.inf))
                continue
            dh = np.abs(h_o[:-1] - h_s[:-1]) / h_s[:-1] if h_o.size > 1 else np.zeros(1)
            res.append((True, int(rec["n_att"][k]) == int(att_s), float(dh.max())))
    return res, rejected


def test_initial_step_equals_scipy_select_initial_step():
    for name in ("lorenz", "vdp"):
        for rtol in (1e-3, 1e-6, 1e-9):
            wl = W.make(name, 16, rtol=rtol, seed=5)
            for k in range(16):
                p, y0 = wl["params"][k], wl["y0"][k]
                f = _rhs(name, p)
                for order in (2, 5, 7):
                    ref = select_initial_step(f, wl["t0"], y0, wl["t1"], np.inf, f(wl["t0"], y0), 1.0, order,
                                              wl["rtol"], wl["atol"])
                    got = oracle.initial_step(name, p, y0, wl["t0"], wl["t1"], wl["rtol"], wl["atol"], order=order)
                    assert abs(got - ref) <= H0_RTOL * ref, (name, rtol, k, order, got, ref)


def test_initial_step_special_cases_equal_scipy():
    # y0 = 0 (d0 < 1e-5: the 1e-6 first guess) and a short span (the interval clamp)
    p = np.array([10.0, 28.0, 8.0 / 3.0])
    f = _rhs("lorenz", p)
    for y0, t1 in ((np.zeros(3), 1.0), (np.array([1.0, 1.0, 1.0]), 1e-7), (np.array([1e-7, 0.0, 0.0]), 1.0)):
        ref = select_initial_step(f, 0.0, y0, t1, np.inf, f(0.0, y0), 1.0, 5, 1e-6, 1e-8)
        got = oracle.initial_step("lorenz", p, y0, 0.0, t1, 1e-6, 1e-8, order=5)
        assert abs(got - ref) <= H0_RTOL * ref, (y0, t1, got, ref)


def test_accepted_mesh_equals_scipy_rk_driver_with_tsit5_table():
    res, rejected = _compare_meshes(_cases())
    same_s = np.mean([r[0] for r in res])
    same_att = np.mean([r[1] for r in res])
    worst = max(r[2] for r in res)
    assert rejected >= 20, rejected  # the cases exercise the rejection path and its cap
    assert same_s == 1.0 and same_att == 1.0, (same_s, same_att)
    assert worst <= H_RTOL, worst


def test_verner7_accepted_mesh_equals_scipy_rk_driver_with_verner_table():
    res, rejected = _compare_meshes(_cases(VERN7), VERN7)
    same = all(r[0] and r[1] for r in res)
    worst = max(r[2] for r in res)
    assert rejected >= 50, rejected
    assert same, [i for i, r in enumerate(res) if not (r[0] and r[1])]
    assert worst <= H_RTOL_V7, worst


# ----------------------------------------------------------------------------- planted mistakes

@contextlib.contextmanager
def _mutant_oracle(old, new):
    """The oracle with one source substitution, compiled like the real one and
    swapped in for the duration of the block."""
    src = open(oracle._SRC).read()
    assert src.count(old) >= 1, old
    d = tempfile.mkdtemp(prefix="oracle_mutant_")
    cpp, so = os.path.join(d, "m.cpp"), os.path.join(d, "m.so")
    with open(cpp, "w") as fh:
        fh.write(src.replace(old, new))
    subprocess.run(["g++", "-O2", "-ffp-contract=off", "-std=c++17", "-fPIC", "-shared", "-o", so, cpp,
                    "-lpthread"], check=True)
    saved = (oracle._lib, oracle._LIB_PATH)
    oracle._lib, oracle._LIB_PATH = None, so
    try:
        yield
    finally:
        oracle._lib, oracle._LIB_PATH = saved


MUTANTS = [
    # starting step: exponent 1/p instead of 1/(p+1)
    ("std::pow(0.01 / dm, 1.0 / (order + 1))", "std::pow(0.01 / dm, 1.0 / order)"),
    # controller exponent -1/q instead of -1/(q+1)
    ("std::pow(err, -1.0 / (q + 1))", "std::pow(err, -1.0 / q)"),
    # safety factor
    ("double f = 0.9 * std::pow", "double f = 0.95 * std::pow"),
    # growth clamp
    ("return std::min(10.0, std::max(0.2, f));", "return std::min(5.0, std::max(0.2, f));"),
    # no cap after a rejection
    ("if (reject_prev) fac = std::min(fac, 1.0);", "(void)reject_prev;"),
    # error scale from |y| only
    ("std::max(std::fabs(y[c]), std::fabs(yn[c]))", "std::fabs(y[c])"),
]


@pytest.mark.parametrize("old,new", MUTANTS)
def test_planted_control_mistake_fails_the_scipy_pins(old, new):
    cases = _cases()[:3]
    with _mutant_oracle(old, new):
        res, _ = _compare_meshes(cases)
        worst = max(r[2] for r in res)
        mesh_ok = all(r[0] and r[1] for r in res) and worst <= H_RTOL
        wl = W.make("lorenz", 4, seed=5)
        f = _rhs("lorenz", wl["params"][0])
        ref = select_initial_step(f, 0.0, wl["y0"][0], 1.0, np.inf, f(0.0, wl["y0"][0]), 1.0, 5, wl["rtol"],
                                  wl["atol"])
        h0 = oracle.initial_step("lorenz", wl["params"][0], wl["y0"][0], 0.0, 1.0, wl["rtol"], wl["atol"], order=5)
        h0_ok = abs(h0 - ref) <= H0_RTOL * ref
    assert not (mesh_ok and h0_ok), f"planted mistake not detected: {new}"


VERN7_MUTANTS = [
    # Verner7's controller exponent from its solution order (-1/8) instead of its estimate's (-1/7)
    ("method == M_VERN7 ? 6 : 4", "method == M_VERN7 ? 7 : 4"),
    # Verner7's starting step with the estimate's order 6 instead of the solution's 7
    ("method == M_VERN7 ? 7 : 5", "method == M_VERN7 ? 6 : 5"),
]


@pytest.mark.parametrize("old,new", VERN7_MUTANTS)
def test_planted_verner7_control_mistake_fails_the_scipy_pin(old, new):
    with _mutant_oracle(old, new):
        res, _ = _compare_meshes(_cases(VERN7)[:2], VERN7)
    worst = max(r[2] for r in res)
    assert not (all(r[0] and r[1] for r in res) and worst <= H_RTOL_V7), f"planted mistake not detected: {new}"


# ----------------------------------------------------------------------------- Rosenbrock methods

def _ros_scipy_mesh(name, method, p, y0, t0, t1, rtol, atol):
    """Accepted steps of scipy's RK driver stepping with the oracle's Rosenbrock step."""
    import scipy.integrate._ivp.rk as rkmod
    order, err_order = (2, 2) if method == ROS23 else (5, 4)
    last = {}

    def fun(t, y):
        return oracle.rhs(name, p, y)[0][0]

    class RosenbrockScipy(RungeKutta):
        C, A, B, E, P = np.zeros(1), np.zeros((1, 1)), np.ones(1), np.zeros(2), np.zeros((2, 1))
        n_stages = 1

        def __init__(self, f, t0_, y0_, t_bound, **kw):
            self.order, self.error_estimator_order = order, err_order
            super().__init__(f, t0_, y0_, t_bound, **kw)
            self.h_abs = select_initial_step(self.fun, self.t, self.y, t_bound, np.inf, self.f, self.direction,
                                             order, self.rtol, self.atol)

        def _estimate_error_norm(self, K, h, scale):
            return float(np.sqrt(np.mean((last["e"] / scale) ** 2)))

    def one_step(f_, t, y, f0, h, A, B, C, K):
        yn, e = oracle.step(name, method, p, y, h)
        last["e"] = e[0]
        K[-1] = fun(t + h, yn[0])
        return yn[0], K[-1]

    saved = rkmod.rk_step
    rkmod.rk_step = one_step
    try:
        sol = solve_ivp(fun, (t0, t1), np.array(y0, dtype=np.float64), method=RosenbrockScipy, rtol=rtol, atol=atol)
    finally:
        rkmod.rk_step = saved
    assert sol.status == 0, sol.message
    return np.diff(sol.t)


def _compare_ros(cases):
    res, rejected = [], 0
    for name, method, wl in cases:
        rec = oracle.record(name, wl["params"], wl["y0"], wl["t0"], wl["t1"], [], wl["rtol"], wl["atol"],
                            method=method, want_saves=False)
        for k in range(wl["params"].shape[0]):
            h_o = rec["h"][rec["offsets"][k]:rec["offsets"][k + 1]]
            h_s = _ros_scipy_mesh(name, method, wl["params"][k], wl["y0"][k], wl["t0"], wl["t1"], wl["rtol"],
                                  wl["atol"])
            rejected += int(rec["n_att"][k] - rec["S"][k])
            if h_o.size != h_s.size:
                res.append((False, np.inf))
                continue
            dh = np.abs(h_o[:-1] - h_s[:-1]) / h_s[:-1] if h_o.size > 1 else np.zeros(1)
            res.append((True, float(dh.max())))
    return res, rejected


def _ros_cases(which=("ros23", "rodas5p")):
    out = []
    if "ros23" in which:
        out += [("robertson", ROS23, W.make("robertson", 8, seed=3)), ("vdp", ROS23, W.make("vdp", 8, seed=3))]
    if "rodas5p" in which:
        out += [("robertson", RODAS5P, W.make("robertson", 8, seed=3)), ("hires", RODAS5P, W.make("hires", 8, seed=3))]
    return out


def test_rosenbrock_meshes_equal_scipy_driver_with_the_oracle_step():
    res, rejected = _compare_ros(_ros_cases())
    assert rejected >= 50, rejected
    assert all(r[0] for r in res), [i for i, r in enumerate(res) if not r[0]]
    assert max(r[1] for r in res) <= H_RTOL_ROS, max(r[1] for r in res)


ROS_MUTANTS = [
    # Rosenbrock23's controller exponent -1/4 instead of -1/3
    ("method == M_ROS23 ? 2 : (method == M_VERN7 ? 6 : 4)", "method == M_ROS23 ? 3 : (method == M_VERN7 ? 6 : 4)",
     "ros23"),
    # Rodas5P's (and Tsit5's) controller exponent -1/6 instead of -1/5
    ("method == M_ROS23 ? 2 : (method == M_VERN7 ? 6 : 4)", "method == M_ROS23 ? 2 : (method == M_VERN7 ? 6 : 5)",
     "rodas5p"),
]


@pytest.mark.parametrize("old,new,which", ROS_MUTANTS)
def test_planted_rosenbrock_control_mistake_fails_the_scipy_pin(old, new, which):
    with _mutant_oracle(old, new):
        res, _ = _compare_ros(_ros_cases((which,))[:1])
    assert not (all(r[0] for r in res) and max(r[1] for r in res) <= H_RTOL_ROS), f"not detected: {new}"
