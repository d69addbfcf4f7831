"""The FP64 step-control form (GS_CONTROL_FP64) of the Tsit5 record.

With the error norm, the accept test, the controller and the starting step in
FP64 (paper Sec. 2.1's weighted RMS norm, accept when it is at most one, the
integral controller; the starting step of Hairer, Norsett & Wanner I, II.4),
the GPU's record follows the oracle's own record: the same accepted and
attempted step counts and the same h up to the rounding of the two codes'
stage sums, which the error estimate's cancellation raises to ~1e-7 in err and
compounds over the steps (the oracle itself agrees with scipy's driver to
5e-8, tests/test_oracle_record_scipy.py). Gradients stay exact on the GPU's
mesh (parity 1e-11 against the oracle replayed there), and the FP32-mixed form
with FP64 control, the precision form with FP64 step control and error norms,
keeps the FP32 parity bound of the fast-control form.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2609_02876_gb300 import _native as N
from paper_2609_02876_gb300 import api
from paper_2609_02876_gb300 import workloads as W
from tests.test_gpu_tsit5 import FP32_MIXED_BOUND, assert_close, dev, fp32_mixed_errors, oracle_on_gpu_mesh, record, \
    reverse

pytestmark = pytest.mark.gpu
H_RTOL = 1e-6


def _mesh_stats(wl, rec):
    off, h = rec.export_mesh()
    orec = oracle.record(wl["problem"], wl["params"], wl["y0"], wl["t0"], wl["t1"], wl["save_t"], wl["rtol"],
                         wl["atol"], want_saves=False)
    same = np.diff(off) == orec["S"]
    worst = 0.0
    for k in np.nonzero(same)[0]:
        a = h[off[k]:off[k + 1]]
        b = orec["h"][orec["offsets"][k]:orec["offsets"][k + 1]]
        worst = max(worst, float((np.abs(a - b) / b)[:-1].max()) if a.size > 1 else 0.0)
    return same.mean(), worst, orec


@pytest.mark.parametrize("name,n,rtol", [("lorenz", 2048, 1e-6), ("lorenz", 1024, 1e-8), ("vdp", 1024, 1e-6)])
def test_fp64_control_mesh_follows_the_oracle(name, n, rtol):
    wl = W.make(name, n, rtol=rtol)
    rec, _, st = record(wl, control="fp64", want_saves=False)
    assert (st.cpu().numpy() == 0).all()
    frac, worst, orec = _mesh_stats(wl, rec)
    att = rec.stats()["attempted"]
    assert frac >= 0.995, frac
    assert worst <= H_RTOL, worst
    assert abs(att - orec["n_att"].sum()) <= 0.005 * att
    # the gradient is exact on the GPU's mesh
    g = reverse(rec, wl)
    o, _, _ = oracle_on_gpu_mesh(wl, rec)
    assert_close(g["params_bar"].T, o["params_bar"], "params_bar")
    assert_close(g["y0_bar"].T, o["y0_bar"], "y0_bar")
    rec.free()


def test_fast_control_mesh_statistics():
    """The default (fast) control evaluates the controller factor in FP32: its
    mesh follows the oracle's more loosely (these bounds are the statistics the
    benchmark reports, with headroom)."""
    wl = W.make("lorenz", 2048)
    rec, _, _ = record(wl, want_saves=False)
    frac, worst, _ = _mesh_stats(wl, rec)
    assert frac >= 0.9, frac
    assert worst <= 1e-4, worst
    rec.free()


def test_fp64_control_solve_grad_matches_record_and_reverse():
    wl = W.make("lorenz", 4096)
    P, Y = dev(wl["params"].T), dev(wl["y0"].T)
    s = api.solve_grad("lorenz", P, Y, wl["t0"], wl["t1"], wl["save_t"], wl["rtol"], wl["atol"], layout="soa",
                       control="fp64")
    rec, _, _ = api.forward_record("lorenz", P, Y, wl["t0"], wl["t1"], wl["save_t"], wl["rtol"], wl["atol"],
                                   layout="soa", want_saves=False, control="fp64", step_counts=True)
    g = api.reverse(rec, P, Y, layout="soa")
    # stored-stage and compact layouts give the same gradient bit for bit
    torch.testing.assert_close(s["params_bar"], g["params_bar"], rtol=0, atol=0)
    torch.testing.assert_close(s["y0_bar"], g["y0_bar"], rtol=0, atol=0)
    f = api.solve("lorenz", P, Y, wl["t0"], wl["t1"], wl["save_t"], wl["rtol"], wl["atol"], layout="soa",
                  control="fp64", step_counts=True)
    np.testing.assert_array_equal(f["step_counts"].cpu().numpy(), rec.step_counts.cpu().numpy())
    rec.free()


@pytest.mark.parametrize("name", ["lorenz", "vdp"])
def test_fp32_mixed_with_fp64_control(name):
    """FP32 stages and adjoint, FP64 error norm and controller: the gradient
    against the FP64 oracle on the run's own mesh stays within the FP32-mixed
    bound of the fast-control form."""
    wl = W.make(name, 1024)
    rec, _, st = record(wl, precision="fp32_mixed", control="fp64", want_saves=False)
    assert (st.cpu().numpy() == 0).all()
    g = reverse(rec, wl)
    o, _, _ = oracle_on_gpu_mesh(wl, rec)
    e = fp32_mixed_errors(g["params_bar"].T, g["y0_bar"].T, o)
    med, mx = FP32_MIXED_BOUND[name]
    assert np.median(e) <= med and e.max() <= mx, (np.median(e), e.max())
    rec.free()


def test_fp64_control_rejects_other_methods_and_shared_weights():
    wl = W.make("lorenz", 8)
    with pytest.raises(N.GsError) as ei:
        record(wl, control="fp64", method="verner7")
    assert ei.value.code == N.GS_ERR_INVALID_ARG
    u = W.make("lv_ude", 8)
    sw = torch.as_tensor(np.asarray(u["w"], dtype=np.float32), device="cuda")
    with pytest.raises(N.GsError) as ei:
        api.solve_grad("lv_ude", dev(u["params"].T), dev(u["y0"].T), u["t0"], u["t1"], u["save_t"], u["rtol"],
                       u["atol"], layout="soa", shared_w=sw, precision="fp32_mixed", control="fp64")
    assert ei.value.code == N.GS_ERR_INVALID_ARG
