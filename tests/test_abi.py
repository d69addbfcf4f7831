"""The C-ABI library builds, loads, exports every symbol include/gs.h declares,
and rejects invalid arguments before touching a GPU (no compute calls here)."""
import ctypes as C

import numpy as np
import pytest

from paper_2609_02876_gb300 import _native as N
from paper_2609_02876_gb300 import build


@pytest.fixture(scope="module")
def lib():
    build.build()
    return N.lib()


def test_exports_every_declared_symbol(lib):
    syms = N.header_symbols()
    assert len(syms) >= 10
    for s in syms:
        assert hasattr(lib, s), f"missing export {s}"


def test_host_only_entry_points(lib):
    assert lib.gs_status_string(0) == b"ok"
    assert b"traj_status" in lib.gs_status_string(5)
    o = N.GsOptions()
    assert lib.gs_default_options(C.byref(o)) == 0
    assert (o.precision, o.method, o.ckpt_k, o.max_steps, o.h0) == (0, 0, 0, 0, 0.0)
    d, P, s, nw = C.c_int(), C.c_int(), C.c_int(), C.c_int()
    expect = {0: (3, 3, 0, 0), 1: (2, 1, 0, 0), 2: (3, 3, 1, 0), 3: (8, 12, 1, 0), 4: (2, 4, 0, 0),
              5: (2, 2, 0, 354), 6: (3, 2, 1, 353)}
    for pid, e in expect.items():
        assert lib.gs_problem_info(pid, C.byref(d), C.byref(P), C.byref(s), C.byref(nw)) == 0
        assert (d.value, P.value, s.value, nw.value) == e
    assert lib.gs_problem_info(17, C.byref(d), C.byref(P), C.byref(s), C.byref(nw)) == N.GS_ERR_UNKNOWN_PROBLEM


def _call(lib, **kw):
    a = dict(pid=0, n=4, params=1, y0=1, w=None, t0=0.0, t1=1.0, save=[0.5, 1.0], rtol=1e-6, atol=1e-8, opt=None)
    a.update(kw)
    st = np.asarray(a["save"], dtype=np.float64)
    o = None
    if a["opt"] is not None:
        o = N.GsOptions()
        lib.gs_default_options(C.byref(o))
        for k, v in a["opt"].items():
            setattr(o, k, v)
        o = C.byref(o)
    return lib.gs_solve_grad(a["pid"], a["n"], a["params"], a["y0"], a["w"], a["t0"], a["t1"],
                             st.ctypes.data_as(C.POINTER(C.c_double)), st.size, a["rtol"], a["atol"], o, None,
                             1, 1, 1, None, 1)


@pytest.mark.parametrize("kw,code", [
    (dict(pid=42), N.GS_ERR_UNKNOWN_PROBLEM),
    (dict(n=-1), N.GS_ERR_INVALID_ARG),
    (dict(params=None), N.GS_ERR_INVALID_ARG),
    (dict(t1=0.0), N.GS_ERR_INVALID_ARG),
    (dict(t1=float("nan")), N.GS_ERR_INVALID_ARG),
    (dict(save=[0.5, 0.5]), N.GS_ERR_INVALID_ARG),
    (dict(save=[0.0]), N.GS_ERR_INVALID_ARG),
    (dict(save=[1.5]), N.GS_ERR_INVALID_ARG),
    (dict(rtol=0.0, atol=0.0), N.GS_ERR_INVALID_ARG),
    (dict(rtol=-1e-6), N.GS_ERR_INVALID_ARG),
    (dict(pid=5), N.GS_ERR_INVALID_ARG),  # the UDE needs shared weights
    (dict(opt=dict(precision=7)), N.GS_ERR_INVALID_ARG),
    (dict(opt=dict(ckpt_k=33)), N.GS_ERR_INVALID_ARG),
    (dict(opt=dict(max_steps=-2)), N.GS_ERR_INVALID_ARG),
    (dict(opt=dict(method=9)), N.GS_ERR_INVALID_ARG),
    (dict(opt=dict(timeout_ms=-1.0)), N.GS_ERR_INVALID_ARG),
    (dict(pid=5, w=1, opt=dict(precision=0)), N.GS_ERR_INVALID_ARG),  # the UDE runs FP32-mixed only
    (dict(pid=0, opt=dict(method=2)), N.GS_ERR_INVALID_ARG),  # no Rodas5P kernel for Lorenz
    (dict(pid=1, opt=dict(method=3)), N.GS_ERR_INVALID_ARG),  # no Rosenbrock23 kernel for Van der Pol
    (dict(pid=2, opt=dict(method=3, precision=1)), N.GS_ERR_INVALID_ARG),  # Rosenbrock23 runs in FP64
    (dict(opt=dict(method=5)), N.GS_ERR_INVALID_ARG),
    (dict(pid=2, opt=dict(method=4)), N.GS_ERR_INVALID_ARG),  # no Verner7 kernel for Robertson
    (dict(pid=0, opt=dict(method=4, precision=1)), N.GS_ERR_INVALID_ARG),  # Verner7 runs in FP64
    (dict(pid=6), N.GS_ERR_INVALID_ARG),  # the neural Robertson needs shared weights
    (dict(pid=6, w=1, opt=dict(precision=1)), N.GS_ERR_INVALID_ARG),  # stiff: FP64 only
    (dict(pid=6, w=1, opt=dict(method=1)), N.GS_ERR_INVALID_ARG),  # no Tsit5 kernel for it
    (dict(pid=6, w=1, opt=dict(ckpt_k=4)), N.GS_ERR_INVALID_ARG),  # shared weights: every state stored
    (dict(opt=dict(control=2)), N.GS_ERR_INVALID_ARG),  # no such step control
    (dict(pid=2, opt=dict(control=1)), N.GS_ERR_INVALID_ARG),  # FP64 step control: Tsit5 only
    (dict(pid=0, opt=dict(control=1, method=4)), N.GS_ERR_INVALID_ARG),  # ... not Verner7
    (dict(pid=5, w=1, opt=dict(control=1, precision=1)), N.GS_ERR_INVALID_ARG),  # ... nor shared weights
    (dict(opt=dict(record_stages=2)), N.GS_ERR_INVALID_ARG),
])
def test_invalid_arguments_are_rejected_on_the_host(lib, kw, code):
    assert _call(lib, **kw) == code


def test_too_many_save_times(lib):
    assert _call(lib, save=np.linspace(0.001, 1.0, 257)) == N.GS_ERR_INVALID_ARG


def test_empty_ensemble_is_a_no_op(lib):
    assert _call(lib, n=0, params=None, y0=None) == N.GS_OK


def _call_solve(lib, **kw):
    a = dict(pid=0, n=4, params=1, y0=1, w=None, t0=0.0, t1=1.0, save=[0.5, 1.0], rtol=1e-6, atol=1e-8,
             y_final=1, status=1)
    a.update(kw)
    st = np.asarray(a["save"], dtype=np.float64)
    return lib.gs_solve(a["pid"], a["n"], a["params"], a["y0"], a["w"], a["t0"], a["t1"],
                        st.ctypes.data_as(C.POINTER(C.c_double)), st.size, a["rtol"], a["atol"], None, None,
                        None, a["y_final"], a["status"])


@pytest.mark.parametrize("kw,code", [
    (dict(pid=42), N.GS_ERR_UNKNOWN_PROBLEM),
    (dict(n=-1), N.GS_ERR_INVALID_ARG),
    (dict(y0=None), N.GS_ERR_INVALID_ARG),
    (dict(t1=-1.0), N.GS_ERR_INVALID_ARG),
    (dict(save=[0.7, 0.2]), N.GS_ERR_INVALID_ARG),
    (dict(y_final=None), N.GS_ERR_INVALID_ARG),
    (dict(status=None), N.GS_ERR_INVALID_ARG),
])
def test_forward_only_solve_rejects_invalid_arguments(lib, kw, code):
    assert _call_solve(lib, **kw) == code


def test_forward_only_solve_of_an_empty_ensemble_is_a_no_op(lib):
    assert _call_solve(lib, n=0, params=None, y0=None, y_final=None, status=None) == N.GS_OK


def test_forward_mode_entry_points_reject_invalid_arguments(lib):
    assert lib.gs_replay_jvp(None, 1, 1, 1, None, None, None, 1, None, None) == N.GS_ERR_INVALID_ARG
    assert lib.gs_forward_grad(None, 1, 1, None, 1, None, None) == N.GS_ERR_INVALID_ARG


def _call_host(lib, **kw):
    a = dict(pid=0, n=4, params=1, y0=1, w=None, t0=0.0, t1=1.0, save=[0.5, 1.0], rtol=1e-6, atol=1e-8, opt=None,
             chunk=0, status=1)
    a.update(kw)
    st = np.asarray(a["save"], dtype=np.float64)
    return lib.gs_solve_grad_host(a["pid"], a["n"], a["params"], a["y0"], a["w"], a["t0"], a["t1"],
                                  st.ctypes.data_as(C.POINTER(C.c_double)), st.size, a["rtol"], a["atol"], a["opt"],
                                  a["chunk"], None, None, None, None, a["status"])


def _opts_with_counts():
    o = N.GsOptions()
    lib_ = N.lib()
    lib_.gs_default_options(C.byref(o))
    o.step_counts = 1
    _opts_with_counts.keep = o
    return C.byref(o)


@pytest.mark.parametrize("kw,code", [
    (dict(pid=42), N.GS_ERR_UNKNOWN_PROBLEM),
    (dict(n=-1), N.GS_ERR_INVALID_ARG),
    (dict(params=None), N.GS_ERR_INVALID_ARG),
    (dict(save=[1.5]), N.GS_ERR_INVALID_ARG),
    (dict(chunk=-2), N.GS_ERR_INVALID_ARG),
    (dict(status=None), N.GS_ERR_INVALID_ARG),
    (dict(pid=6), N.GS_ERR_INVALID_ARG),  # the neural Robertson needs its shared weights
])
def test_host_buffer_entry_rejects_invalid_arguments(lib, kw, code):
    assert _call_host(lib, **kw) == code


def test_host_buffer_entry_rejects_device_step_counts_and_empty_is_a_no_op(lib):
    assert _call_host(lib, opt=_opts_with_counts()) == N.GS_ERR_INVALID_ARG
    assert _call_host(lib, n=0, params=None, y0=None, status=None) == N.GS_OK
