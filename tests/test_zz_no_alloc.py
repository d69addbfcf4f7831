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


def _noalloc(L, wl, P, Y):
    n = P.shape[1]
    d = Y.shape[0]
    out = {"loss": torch.full((n,), float("nan"), dtype=torch.float64, device="cuda"),
           "params_bar": torch.full((P.shape[0], n), float("nan"), dtype=torch.float64, device="cuda"),
           "y0_bar": torch.full((d, n), float("nan"), dtype=torch.float64, device="cuda"),
           "status": torch.full((n,), -1, dtype=torch.int32, device="cuda")}
    st = np.ascontiguousarray(wl["save_t"], dtype=np.float64)
    rc = L.gs_solve_grad_noalloc(N.PROBLEMS[wl["problem"]], n, P.data_ptr(), Y.data_ptr(), None, wl["t0"],
                                 wl["t1"], st.ctypes.data_as(C.POINTER(C.c_double)), st.size, wl["rtol"],
                                 wl["atol"], None, torch.cuda.current_stream().cuda_stream,
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
