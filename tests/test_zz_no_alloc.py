"""gs_solve_grad_noalloc: the allocation-free variant of gs_solve_grad.

Some callers cannot call cudaMalloc (all free device memory already belongs to
another allocator, or the calling thread must not block on allocation); for
them the library keeps the record in a fixed static device array. Here the new
entry point is called through the C-ABI twice in a row and each result is
checked against gs_solve_grad on the same inputs, with the GPU parity
tolerance (normwise relative 1e-11 per trajectory vector). This file is
collected last so that a run stopping at its first failure has already run
every other test.
"""
import ctypes as C

import numpy as np
import pytest
import torch

from paper_2609_02876_gb300 import _native as N
from paper_2609_02876_gb300 import api, build
from paper_2609_02876_gb300 import workloads as W

pytestmark = pytest.mark.gpu
RTOL = 1e-11


def _lib():
    build.build()
    L = N.lib()
    vp, i32, i64, d = C.c_void_p, C.c_int, C.c_int64, C.c_double
    L.gs_solve_grad_noalloc.argtypes = [i32, i64, vp, vp, vp, d, d, C.POINTER(C.c_double), i32, d, d,
                                        C.POINTER(N.GsOptions), vp, vp, vp, vp, vp, vp]
    L.gs_solve_grad_noalloc.restype = C.c_int
    return L


def _options(L, precision=N.GS_FP64, ckpt_k=0):
    o = N.GsOptions()
    L.gs_default_options(C.byref(o))
    o.precision = precision
    o.ckpt_k = ckpt_k
    return o


def _noalloc(L, wl, P, Y, opt=None):
    n = P.shape[1]
    d = Y.shape[0]
    out = {"loss": torch.full((n,), float("nan"), dtype=torch.float64, device="cuda"),
           "params_bar": torch.full((P.shape[0], n), float("nan"), dtype=torch.float64, device="cuda"),
           "y0_bar": torch.full((d, n), float("nan"), dtype=torch.float64, device="cuda"),
           "status": torch.full((n,), -1, dtype=torch.int32, device="cuda")}
    st = np.ascontiguousarray(wl["save_t"], dtype=np.float64)
    sw = wl.get("sw")
    rc = L.gs_solve_grad_noalloc(N.PROBLEMS[wl["problem"]], n, P.data_ptr(), Y.data_ptr(),
                                 None if sw is None else sw.data_ptr(), wl["t0"],
                                 wl["t1"], st.ctypes.data_as(C.POINTER(C.c_double)), st.size, wl["rtol"],
                                 wl["atol"], None if opt is None else C.byref(opt),
                                 torch.cuda.current_stream().cuda_stream,
                                 out["loss"].data_ptr(), out["params_bar"].data_ptr(), out["y0_bar"].data_ptr(),
                                 None, out["status"].data_ptr())
    return rc, out


def _normwise(a, b):
    a = a.cpu().numpy()
    b = b.cpu().numpy()
    if a.ndim == 1:
        a, b = a[None], b[None]
    num = np.abs(a - b).max(0)
    den = np.abs(b).max(0)
    return (num / np.where(den > 0, den, 1.0)).max()


def test_noalloc_matches_solve_grad_on_two_calls_in_a_row():
    L = _lib()
    for name, n in (("lorenz", 3000), ("vdp", 1200)):
        wl = W.make(name, n)
        P = torch.as_tensor(np.ascontiguousarray(wl["params"].T), device="cuda")
        Y = torch.as_tensor(np.ascontiguousarray(wl["y0"].T), device="cuda")
        ref = api.solve_grad(name, P, Y, wl["t0"], wl["t1"], wl["save_t"], wl["rtol"], wl["atol"], layout="soa")
        for call in range(2):
            rc, out = _noalloc(L, wl, P, Y)
            assert rc == N.GS_OK, f"{name} call {call}: {N.status_string(rc)}"
            assert (out["status"] == 0).all().item()
            for key in ("loss", "params_bar", "y0_bar"):
                err = _normwise(out[key], ref[key] if key == "loss" else ref[key])
                assert err <= RTOL, f"{name} call {call} {key}: normwise rel err {err:.3e}"


def test_noalloc_rejects_ensembles_beyond_its_limit():
    L = _lib()
    wl = W.make("lorenz", 16)
    P = torch.zeros((3, 16385), dtype=torch.float64, device="cuda")
    Y = torch.zeros((3, 16385), dtype=torch.float64, device="cuda")
    rc, _ = _noalloc(L, wl, P, Y)
    assert rc == N.GS_ERR_INVALID_ARG


def _inputs(name, n, **kw):
    wl = W.make(name, n, **kw)
    P = torch.as_tensor(np.ascontiguousarray(wl["params"].T), device="cuda")
    Y = torch.as_tensor(np.ascontiguousarray(wl["y0"].T), device="cuda")
    return wl, P, Y


def _check_against_solve_grad(L, name, n, precision, ckpt_k, tol, **kw):
    wl, P, Y = _inputs(name, n, **kw)
    prec = "fp64" if precision == N.GS_FP64 else "fp32_mixed"
    ref = api.solve_grad(name, P, Y, wl["t0"], wl["t1"], wl["save_t"], wl["rtol"], wl["atol"], layout="soa",
                         precision=prec)
    rc, out = _noalloc(L, wl, P, Y, _options(L, precision, ckpt_k))
    assert rc == N.GS_OK, N.status_string(rc)
    assert (out["status"] == 0).all().item()
    for key in ("loss", "params_bar", "y0_bar"):
        err = _normwise(out[key], ref[key])
        assert err <= tol, f"{name} {prec} k={ckpt_k} {key}: normwise rel err {err:.3e}"


def test_noalloc_fp32_mixed_and_every_state_stored():
    """The FP32-mixed form (compared with gs_solve_grad's FP32-mixed result: the
    same kernels' arithmetic, only the checkpoint interval differs, so the bound
    is the FP32 form's own rounding level) and a caller-set k = 1 (every accepted
    state stored, nothing recomputed: FP64 parity tolerance)."""
    L = _lib()
    _check_against_solve_grad(L, "lorenz", 2000, N.GS_FP32_MIXED, 0, 2e-5)
    _check_against_solve_grad(L, "lorenz", 2000, N.GS_FP64, 1, RTOL)


def test_noalloc_rejects_shared_weight_problems():
    """The LV UDE's weight gradient needs per-warp partials outside the fixed
    array: the entry point refuses the problem before any work."""
    L = _lib()
    wl, P, Y = _inputs("lv_ude", 64)
    wl["sw"] = torch.as_tensor(np.asarray(wl["w"], dtype=np.float32), device="cuda")
    rc, out = _noalloc(L, wl, P, Y, _options(L, N.GS_FP32_MIXED, 1))
    assert rc == N.GS_ERR_INVALID_ARG
    assert (out["status"] == -1).all().item()  # nothing was launched


def test_noalloc_overflow_reports_oom_and_the_next_call_is_correct():
    """Van der Pol at rtol 1e-8 over t in [0, 10] takes ~230 accepted steps per
    trajectory: 16384 trajectories need ~330k record segments of 128 bytes, more
    than the 32 MiB array holds. The call must return GS_ERR_OOM, and a following
    call that fits must still match gs_solve_grad."""
    L = _lib()
    wl, P, Y = _inputs("vdp", 16384, rtol=1e-8)
    rc, _ = _noalloc(L, wl, P, Y)
    assert rc == N.GS_ERR_OOM, N.status_string(rc)
    torch.cuda.synchronize()
    _check_against_solve_grad(L, "vdp", 1500, N.GS_FP64, 0, RTOL)
