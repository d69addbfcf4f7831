"""The full-lane passes that run before the persistent kernels give the same
bits as the per-trajectory code they replace.

- The t1-save pass (FP64 k = 1 reverse sweep, last save time t1) writes the
  save's cotangent and loss term into y0_bar and loss, and the sweep starts
  from them. gs_reverse without y0_bar skips the pass and takes that save in
  the sweep itself: params_bar and loss must be bit-identical either way, for
  the compact and the stored-stage record, the built-in loss and a caller's
  cotangent, and for a save grid that does not end at t1 (no pass).
- The starting-step pass before the record is compared the same way in
  tests/test_gpu_solve.py (an in-place gs_solve skips it).
"""
import ctypes as C

import numpy as np
import pytest
import torch

from paper_2609_02876_gb300 import _native as N
from paper_2609_02876_gb300 import api, build
from paper_2609_02876_gb300 import workloads as W
from tests.test_gpu_tsit5 import dev, record

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def _raw_reverse(rec, wl, want_y0_bar, ybar=None):
    n, d, P = rec.n, rec.d, rec.P
    p, y = dev(wl["params"].T), dev(wl["y0"].T)
    pb = torch.empty((P, n), dtype=torch.float64, device="cuda")
    y0b = torch.empty((d, n), dtype=torch.float64, device="cuda") if want_y0_bar else None
    loss = torch.empty(n, dtype=torch.float64, device="cuda") if ybar is None else None
    yb = ybar.contiguous() if ybar is not None else None
    ptr = lambda t: C.c_void_p(t.data_ptr()) if t is not None else None
    rc = N.lib().gs_reverse(rec.handle, ptr(p), ptr(y), None, ptr(yb), ptr(loss), ptr(pb), ptr(y0b), None,
                            C.c_void_p(api._stream()))
    torch.cuda.synchronize()
    assert rc == N.GS_OK, rc
    return pb, y0b, loss


@pytest.mark.parametrize("name,stages,user_cot,save_at_t1",
                         [("lorenz", False, False, True), ("lorenz", True, False, True),
                          ("lorenz", True, True, True), ("vdp", True, False, True),
                          ("robertson", True, False, True), ("lorenz", True, False, False)])
def test_t1_save_pass_is_bit_identical(name, stages, user_cot, save_at_t1):
    wl = W.make(name, 777)
    if not save_at_t1:
        wl = dict(wl, save_t=np.asarray(wl["save_t"])[:-1])
    rec, _, st = record(wl, want_saves=False, ckpt_k=1, record_stages=stages)
    assert (st.cpu().numpy() == 0).all()
    ybar = None
    if user_cot:
        g = torch.Generator().manual_seed(5)
        ybar = torch.randn((len(wl["save_t"]), rec.d, rec.n), generator=g, dtype=torch.float64).cuda()
    pb_a, y0b_a, loss_a = _raw_reverse(rec, wl, True, ybar)
    pb_b, _, loss_b = _raw_reverse(rec, wl, False, ybar)
    assert torch.isfinite(pb_a).all() and torch.isfinite(y0b_a).all()
    assert torch.equal(pb_a, pb_b)
    if loss_a is not None:
        assert torch.equal(loss_a, loss_b)
    rec.free()
