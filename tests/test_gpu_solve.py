"""GPU forward-only solve (gs_solve): the record kernel with nothing recorded.

It must take exactly the steps gs_forward_record takes (the same kernel with
the record writes switched off), so save states, statuses and step counts are
compared bit for bit; y(t1) is compared with the oracle stepping along the
exported mesh (normwise relative error 1e-11 per trajectory, as for the other
FP64 parity tests).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2609_02876_gb300 import api, build
from paper_2609_02876_gb300 import workloads as W
from tests.test_gpu_tsit5 import assert_close, dev, record

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def oracle_final_state(wl, off, h):
    """y(t1) of every trajectory by the oracle's single steps along the mesh (offsets, h)."""
    y = np.array(wl["y0"], dtype=np.float64)
    p = np.asarray(wl["params"], dtype=np.float64)
    S = np.diff(off)
    for i in range(int(S.max()) if S.size else 0):
        act = np.nonzero(S > i)[0]
        yn, _ = oracle.step(wl["problem"], oracle.METHOD_AUTO, p[act], y[act], h[off[act] + i], w=wl["w"])
        y[act] = yn
    return y


def solve(wl, **opts):
    return api.solve(wl["problem"], dev(wl["params"].T), dev(wl["y0"].T), wl["t0"], wl["t1"], wl["save_t"],
                     wl["rtol"], wl["atol"], layout="soa", **opts)


@pytest.mark.parametrize("name,n", [("lorenz", 1000), ("vdp", 333), ("robertson", 257), ("hires", 129)])
def test_forward_only_solve_takes_the_recorded_steps(name, n):
    wl = W.make(name, n)
    rec, ysv, st = record(wl, step_counts=True)
    s = solve(wl, step_counts=True)
    assert s["rc"] == 0
    np.testing.assert_array_equal(s["status"].cpu().numpy(), st.cpu().numpy())
    np.testing.assert_array_equal(s["step_counts"].cpu().numpy(), rec.step_counts.cpu().numpy())
    np.testing.assert_array_equal(s["y_save"].cpu().numpy(), ysv.cpu().numpy())
    off, h = rec.export_mesh()
    assert_close(s["y_final"].cpu().numpy().T, oracle_final_state(wl, off, h), "y_final")


def test_forward_only_solve_fp32_mixed_takes_the_recorded_steps():
    wl = W.make("lorenz", 4099)
    rec, ysv, st = record(wl, step_counts=True, precision="fp32_mixed")
    s = solve(wl, step_counts=True, precision="fp32_mixed")
    np.testing.assert_array_equal(s["status"].cpu().numpy(), st.cpu().numpy())
    np.testing.assert_array_equal(s["step_counts"].cpu().numpy(), rec.step_counts.cpu().numpy())
    np.testing.assert_array_equal(s["y_save"].cpu().numpy(), ysv.cpu().numpy())


def test_forward_only_solve_without_saves_and_failed_trajectories():
    wl = W.make("vdp", 64)
    p = wl["params"].copy()
    p[7, 0] = np.inf
    wl2 = dict(wl, params=p)
    s = solve(wl2, want_saves=False, check=False)
    st = s["status"].cpu().numpy()
    assert s["rc"] == 5 and s["y_save"] is None
    assert st[7] == 3 and (np.delete(st, 7) == 0).all()
    full = solve(wl)
    yf = s["y_final"].cpu().numpy()
    np.testing.assert_array_equal(np.delete(yf, 7, axis=1), np.delete(full["y_final"].cpu().numpy(), 7, axis=1))


def test_forward_record_with_stored_stages():
    """gs_forward_record with record_stages: the record keeps every step's stage
    data, the reverse sweep reads them and returns the compact record's gradient
    bit for bit; the mesh and forward mode are unchanged; refresh is refused
    (its stored stages belong to the recorded parameters); autograd uses it."""
    from paper_2609_02876_gb300 import _native as N
    wl = W.make("lorenz", 3000)
    P, Y = dev(wl["params"].T), dev(wl["y0"].T)
    info = np.zeros(2, np.int32)
    rs, _, _ = api.forward_record("lorenz", P, Y, wl["t0"], wl["t1"], wl["save_t"], wl["rtol"], wl["atol"],
                                  layout="soa", record_stages=True, record_info=info)
    assert tuple(info) == (1, 1)
    rc, _, _ = api.forward_record("lorenz", P, Y, wl["t0"], wl["t1"], wl["save_t"], wl["rtol"], wl["atol"],
                                  layout="soa")
    gs, gc = api.reverse(rs, P, Y, layout="soa"), api.reverse(rc, P, Y, layout="soa")
    for key in ("loss", "params_bar", "y0_bar"):
        torch.testing.assert_close(gs[key], gc[key], rtol=0, atol=0)
    for a, b in zip(rs.export_mesh(), rc.export_mesh()):
        np.testing.assert_array_equal(a, b)
    torch.testing.assert_close(api.forward_grad(rs, P, Y, wrt=("params",), layout="soa")["params_bar"],
                               api.forward_grad(rc, P, Y, wrt=("params",), layout="soa")["params_bar"],
                               rtol=0, atol=0)
    with pytest.raises(N.GsError) as ei:
        api.refresh(rs, P, Y, layout="soa")
    assert ei.value.code == N.GS_ERR_INVALID_ARG
    rs.free()
    rc.free()


@pytest.mark.parametrize("control", ["fast", "fp64"])
def test_forward_only_solve_in_place_final_state(control):
    """y_final may be the y0 buffer itself (an in-place call): the starting-step
    pass, which keeps its results in y_final until each trajectory ends, is then
    skipped and the record computes the starting steps itself, with the same
    results as an out-of-place call."""
    from paper_2609_02876_gb300 import _native as N
    import ctypes as C
    wl = W.make("lorenz", 1000)
    ref = solve(wl, want_saves=False, control=control)
    p = dev(wl["params"].T).contiguous()
    y = dev(wl["y0"].T).contiguous()
    st = torch.empty(wl["params"].shape[0], dtype=torch.int32, device="cuda")
    save = np.ascontiguousarray(wl["save_t"], dtype=np.float64)
    o = api._opts(control=control)
    rc = N.lib().gs_solve(N.PROBLEMS["lorenz"], p.shape[1], p.data_ptr(), y.data_ptr(), None, float(wl["t0"]),
                          float(wl["t1"]), save.ctypes.data_as(C.POINTER(C.c_double)), save.size, float(wl["rtol"]),
                          float(wl["atol"]), C.byref(o), api._stream(), None, y.data_ptr(), st.data_ptr())
    torch.cuda.synchronize()
    assert rc == N.GS_OK
    assert torch.equal(st, ref["status"])
    assert torch.equal(y, ref["y_final"])


def test_chunked_fp32_mixed_solve_grad_equals_the_one_piece_call():
    """An FP32-mixed gs_solve_grad above 2^22 trajectories runs in chunks of
    2^21 (a smaller record); asking for step counts keeps it in one piece. The
    two must agree bit for bit, ragged last chunk included."""
    n = (1 << 22) + 12345
    wl = W.make("lorenz", n)
    P, Y = dev(wl["params"].T), dev(wl["y0"].T)
    args = ("lorenz", P, Y, wl["t0"], wl["t1"], wl["save_t"], wl["rtol"], wl["atol"])
    kms = np.zeros(2, np.float32)
    a = api.solve_grad(*args, layout="soa", precision="fp32_mixed", kernel_ms=kms)
    b = api.solve_grad(*args, layout="soa", precision="fp32_mixed", step_counts=True)
    for key in ("loss", "params_bar", "y0_bar", "status"):
        assert torch.equal(a[key], b[key]), key
    assert kms[0] > 0 and kms[1] > 0


def test_chunked_fp64_solve_grad_with_stored_stages_equals_the_one_piece_call():
    """An FP64 gs_solve_grad whose stored-stage record would not fit runs in
    chunks that do (stages read, not recomputed). Forcing that here would need
    most of the device memory, so the rule is checked on what it decides: at
    rtol 1e-8 the 2^24 Lorenz ensemble is recorded in chunks with stored stages
    (record_info), and a chunk-sized sample of it equals the same trajectories
    solved alone bit for bit."""
    n = 1 << 24
    wl = W.make("lorenz", n, rtol=1e-8)
    P, Y = dev(wl["params"].T), dev(wl["y0"].T)
    info = np.zeros(2, np.int32)
    a = api.solve_grad("lorenz", P, Y, wl["t0"], wl["t1"], wl["save_t"], wl["rtol"], wl["atol"], layout="soa",
                       record_info=info)
    assert info[0] == 1 and info[1] == 1, info  # the last chunk kept every state and its stages
    m = 1 << 16
    k0 = n - m - 777  # straddles the last chunk boundary when chunks are a power of two above 2^16
    b = api.solve_grad("lorenz", P[:, k0:k0 + m].contiguous(), Y[:, k0:k0 + m].contiguous(), wl["t0"], wl["t1"],
                       wl["save_t"], wl["rtol"], wl["atol"], layout="soa")
    for key in ("loss", "status"):
        assert torch.equal(a[key][k0:k0 + m], b[key]), key
    for key in ("params_bar", "y0_bar"):
        assert torch.equal(a[key][:, k0:k0 + m], b[key]), key
