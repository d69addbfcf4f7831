"""Python access to the FP64 CPU oracle (``gs_oracle.cpp``).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` use this module; the product path
(``paper_2609_02876_gb300``) never imports it.

All arrays here are per trajectory (row-major, trajectory-first): params
``(n, P)``, y0 ``(n, d)``, save-time states ``(n, n_save, d)``. The mesh is
ragged: ``h[offsets[k]:offsets[k+1]]`` are trajectory k's accepted step sizes.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gs_oracle.cpp")
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle.so")

PROBLEMS = {"lorenz": 0, "vdp": 1, "robertson": 2, "hires": 3, "linear": 4, "lv_ude": 5, "nrob": 6}
METHOD_AUTO, METHOD_TSIT5, METHOD_RODAS5P, METHOD_ROSENBROCK23, METHOD_VERNER7 = 0, 1, 2, 3, 4
TRAJ_OK, TRAJ_MAXSTEPS, TRAJ_DT_UNDERFLOW, TRAJ_NONFINITE, TRAJ_SINGULAR = 0, 1, 2, 3, 4


def build(force: bool = False) -> str:
    """Compile the oracle with g++ (-O2, no FMA contraction) into oracle/_build."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        cmd = ["g++", "-O2", "-ffp-contract=off", "-std=c++17", "-fPIC", "-shared", "-o", _LIB_PATH, _SRC,
               "-lpthread"]
        subprocess.run(cmd, check=True)
    return _LIB_PATH


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB_PATH)
        dp = C.POINTER(C.c_double)
        lp = C.POINTER(C.c_int64)
        ip = C.POINTER(C.c_int32)
        i32 = C.c_int
        i64 = C.c_int64
        d = C.c_double
        L.or_problem_info.argtypes = [i32, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int),
                                      C.POINTER(C.c_int)]
        L.or_tableau.argtypes = [i32, dp, dp, dp, dp]
        L.or_record.argtypes = [i32, i32, i64, dp, dp, dp, d, d, dp, i32, d, d, i64, d, i64, lp, dp, lp, dp, ip,
                                i32]
        L.or_replay_grad.argtypes = [i32, i32, i64, dp, dp, dp, d, d, dp, i32, lp, dp, dp, dp, dp, dp, dp, dp, ip,
                                     i32]
        L.or_replay_jvp.argtypes = [i32, i32, i64, dp, dp, dp, d, d, dp, i32, lp, dp, dp, dp, dp, dp, dp, i32]
        L.or_step.argtypes = [i32, i32, i64, dp, dp, dp, dp, dp, dp]
        L.or_rhs.argtypes = [i32, i64, dp, dp, dp, dp, dp]
        L.or_initial_step.argtypes = [i32, dp, dp, dp, d, d, d, d, i32]
        L.or_initial_step.restype = C.c_double
        L.or_w_contract.argtypes = [i32, dp, dp, dp, dp, dp]
        _lib = L
    return _lib


def _pid(problem) -> int:
    return PROBLEMS[problem] if isinstance(problem, str) else int(problem)


def _p(a, dtype=np.float64):
    if a is None:
        return None
    return a.ctypes.data_as(C.POINTER(C.c_double if dtype == np.float64 else
                                      (C.c_int64 if dtype == np.int64 else C.c_int32)))


def _arr(x, dtype=np.float64):
    return np.ascontiguousarray(np.asarray(x, dtype=dtype))


def problem_info(problem):
    d, P, s, nw = C.c_int(), C.c_int(), C.c_int(), C.c_int()
    if lib().or_problem_info(_pid(problem), C.byref(d), C.byref(P), C.byref(s), C.byref(nw)) != 0:
        raise ValueError(f"unknown problem {problem}")
    return d.value, P.value, bool(s.value), nw.value


def tableau(method: int):
    if method in (METHOD_TSIT5, METHOD_VERNER7):
        s = 7 if method == METHOD_TSIT5 else 10
        A, b, bh, c = np.zeros(s * s), np.zeros(s), np.zeros(s), np.zeros(s)
        lib().or_tableau(method, _p(A), _p(b), _p(bh), _p(c))
        return {"A": A.reshape(s, s), "b": b, "bhat": bh, "c": c}
    a, m, Cm, g = np.zeros(64), np.zeros(8), np.zeros(64), np.zeros(1)
    lib().or_tableau(method, _p(a), _p(m), _p(Cm), _p(g))
    return {"a": a.reshape(8, 8), "C": Cm.reshape(8, 8), "m": m, "gamma": float(g[0])}


def _w(problem, w):
    if _pid(problem) in (PROBLEMS["lv_ude"], PROBLEMS["nrob"]):
        if w is None:
            raise ValueError("shared-weight problems need their weights")
        return _arr(w)
    return None


def record(problem, params, y0, t0, t1, save_t, rtol, atol, method=METHOD_AUTO, max_steps=10**6, h_init=0.0,
           mesh_cap=1 << 14, w=None, nthreads=0, want_saves=True):
    """Adaptive record per trajectory. Returns dict with offsets, h, S, n_att, status, y_save."""
    pid = _pid(problem)
    d, P, _, _ = problem_info(pid)
    params, y0, save_t = _arr(params).reshape(-1, P), _arr(y0).reshape(-1, d), _arr(save_t).reshape(-1)
    n, ns = params.shape[0], save_t.shape[0]
    w = _w(pid, w)
    S = np.zeros(n, np.int64)
    natt = np.zeros(n, np.int64)
    mesh = np.zeros((n, mesh_cap))
    ysv = np.zeros((n, ns, d)) if want_saves else None
    st = np.zeros(n, np.int32)
    rc = lib().or_record(pid, method, n, _p(params), _p(y0), _p(w), t0, t1, _p(save_t), ns, rtol, atol,
                         int(max_steps), h_init, mesh_cap, _p(S, np.int64), _p(mesh), _p(natt, np.int64),
                         _p(ysv), _p(st, np.int32), nthreads)
    if rc != 0:
        raise RuntimeError(f"or_record failed: {rc}")
    if (S < 0).any():
        raise RuntimeError("mesh_cap too small")
    offsets = np.zeros(n + 1, np.int64)
    offsets[1:] = np.cumsum(S)
    h = np.concatenate([mesh[k, :S[k]] for k in range(n)]) if n else np.zeros(0)
    return {"offsets": offsets, "h": np.ascontiguousarray(h), "S": S, "n_att": natt, "status": st,
            "y_save": ysv}


def replay_grad(problem, params, y0, t0, t1, save_t, offsets, h, ybar_save=None, method=METHOD_AUTO, w=None,
                nthreads=0):
    """Replay on a given mesh plus the discrete adjoint. Returns dict(loss, y_save, params_bar, y0_bar, w_bar, ok)."""
    pid = _pid(problem)
    d, P, _, nw = problem_info(pid)
    params, y0, save_t = _arr(params).reshape(-1, P), _arr(y0).reshape(-1, d), _arr(save_t).reshape(-1)
    n, ns = params.shape[0], save_t.shape[0]
    offsets, h = _arr(offsets, np.int64), _arr(h)
    w = _w(pid, w)
    yb = None if ybar_save is None else _arr(ybar_save).reshape(n, ns, d)
    loss, ysv = np.zeros(n), np.zeros((n, ns, d))
    pb, y0b = np.zeros((n, P)), np.zeros((n, d))
    wb = np.zeros(nw) if nw else None
    ok = np.zeros(n, np.int32)
    rc = lib().or_replay_grad(pid, method, n, _p(params), _p(y0), _p(w), t0, t1, _p(save_t), ns,
                              _p(offsets, np.int64), _p(h), _p(yb), _p(loss), _p(ysv), _p(pb), _p(y0b), _p(wb),
                              _p(ok, np.int32), nthreads)
    if rc != 0:
        raise RuntimeError(f"or_replay_grad failed: {rc}")
    return {"loss": loss, "y_save": ysv, "params_bar": pb, "y0_bar": y0b, "w_bar": wb, "ok": ok.astype(bool)}


def replay_jvp(problem, params, y0, t0, t1, save_t, offsets, h, params_dot, y0_dot, method=METHOD_AUTO, w=None,
               nthreads=0):
    """Dual-number directional derivative of the replay's built-in loss and save states."""
    pid = _pid(problem)
    d, P, _, _ = problem_info(pid)
    params, y0, save_t = _arr(params).reshape(-1, P), _arr(y0).reshape(-1, d), _arr(save_t).reshape(-1)
    n, ns = params.shape[0], save_t.shape[0]
    pdot, ydot = _arr(params_dot).reshape(n, P), _arr(y0_dot).reshape(n, d)
    offsets, h = _arr(offsets, np.int64), _arr(h)
    w = _w(pid, w)
    loss, ldot, ysd = np.zeros(n), np.zeros(n), np.zeros((n, ns, d))
    rc = lib().or_replay_jvp(pid, method, n, _p(params), _p(y0), _p(w), t0, t1, _p(save_t), ns,
                             _p(offsets, np.int64), _p(h), _p(pdot), _p(ydot), _p(loss), _p(ldot), _p(ysd),
                             nthreads)
    if rc != 0:
        raise RuntimeError(f"or_replay_jvp failed: {rc}")
    return {"loss": loss, "loss_dot": ldot, "y_save_dot": ysd}


def step(problem, method, params, y, h, w=None):
    """One step of the method from each y with per-trajectory h. Returns (y_new, err)."""
    pid = _pid(problem)
    d, P, _, _ = problem_info(pid)
    params, y, h = _arr(params).reshape(-1, P), _arr(y).reshape(-1, d), _arr(h).reshape(-1)
    n = y.shape[0]
    yn, e = np.zeros((n, d)), np.zeros((n, d))
    rc = lib().or_step(pid, method, n, _p(params), _p(y), _p(_w(pid, w)), _p(h), _p(yn), _p(e))
    if rc != 0:
        raise RuntimeError(f"or_step failed: {rc}")
    return yn, e


def rhs(problem, params, y, w=None):
    """f(y) and J = df/dy at each point: shapes (n, d), (n, d, d)."""
    pid = _pid(problem)
    d, P, _, _ = problem_info(pid)
    params, y = _arr(params).reshape(-1, P), _arr(y).reshape(-1, d)
    n = y.shape[0]
    f, J = np.zeros((n, d)), np.zeros((n, d, d))
    lib().or_rhs(pid, n, _p(params), _p(y), _p(_w(pid, w)), _p(f), _p(J))
    return f, J


def initial_step(problem, params, y0, t0, t1, rtol, atol, w=None, order=5):
    """Starting step (Hairer-Norsett-Wanner) for a method of the given order (5: Tsit5, Rodas5P; 2: Rosenbrock23)."""
    pid = _pid(problem)
    return lib().or_initial_step(pid, _p(_arr(params)), _p(_arr(y0)), _p(_w(pid, w)), t0, t1, rtol, atol, order)


def solve_grad(problem, params, y0, t0, t1, save_t, rtol, atol, method=METHOD_AUTO, w=None, nthreads=0,
               max_steps=10**6):
    """Record, then the replay gradient on the oracle's own mesh (built-in loss)."""
    rec = record(problem, params, y0, t0, t1, save_t, rtol, atol, method=method, w=w, nthreads=nthreads,
                 max_steps=max_steps, want_saves=False)
    g = replay_grad(problem, params, y0, t0, t1, save_t, rec["offsets"], rec["h"], method=method, w=w,
                    nthreads=nthreads)
    g["record"] = rec
    return g


def w_contract(problem, y, w, r, u):
    """Shared-weight gradient of r^T J(y, w) u at one point (stiff-adjoint contraction term)."""
    pid = _pid(problem)
    _, _, _, nw = problem_info(pid)
    out = np.zeros(nw)
    rc = lib().or_w_contract(pid, _p(_arr(y)), _p(_arr(w)), _p(_arr(r)), _p(_arr(u)), _p(out))
    if rc != 0:
        raise RuntimeError(f"or_w_contract failed: {rc}")
    return out
