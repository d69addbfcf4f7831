"""Conservation-law pins (paper Appendix A).

Robertson conserves y1 + y2 + y3; HIRES conserves y7 + y8. Explicit RK and
Rosenbrock steps preserve linear invariants exactly (up to roundoff), so every
save-time state keeps them; and by the same token the adjoint of the invariant
(cotangent e at one save time) must return y0_bar = e and theta_bar = 0.
"""
import numpy as np
import pytest

import oracle
from paper_2609_02876_gb300 import workloads as W


@pytest.mark.parametrize("name,idx,total", [("robertson", [0, 1, 2], 1.0), ("hires", [6, 7], 0.0057)])
def test_invariant_forward_and_adjoint(name, idx, total):
    wl = W.make(name, 4)
    rec = oracle.record(wl["problem"], wl["params"], wl["y0"], wl["t0"], wl["t1"], wl["save_t"], wl["rtol"],
                        wl["atol"])
    assert (rec["status"] == 0).all()
    inv = rec["y_save"][:, :, idx].sum(-1)
    np.testing.assert_allclose(inv, total, rtol=0, atol=1e-13 * max(1.0, total) + 1e-15)
    e = np.zeros(wl["y0"].shape[1])
    e[idx] = 1.0
    for s in (0, len(wl["save_t"]) // 2, len(wl["save_t"]) - 1):
        ybar = np.zeros_like(rec["y_save"])
        ybar[:, s, :] = e
        g = oracle.replay_grad(wl["problem"], wl["params"], wl["y0"], wl["t0"], wl["t1"], wl["save_t"],
                               rec["offsets"], rec["h"], ybar_save=ybar)
        np.testing.assert_allclose(g["y0_bar"], np.tile(e, (4, 1)), atol=1e-10)
        # theta_bar of a conserved quantity vanishes (relative to the rate scale)
        assert np.all(np.abs(g["params_bar"] * wl["params"]) < 1e-9)


def test_robertson_mass_at_every_mesh_point():
    wl = W.make("robertson", 2)
    rec = oracle.record(wl["problem"], wl["params"], wl["y0"], wl["t0"], wl["t1"], wl["save_t"], wl["rtol"],
                        wl["atol"])
    # one save exactly at every mesh point of trajectory 0: side steps of length 0
    h = rec["h"][: rec["S"][0]]
    ts = [wl["t0"]]
    for i, hi in enumerate(h):
        ts.append(wl["t1"] if i == len(h) - 1 else ts[-1] + hi)
    saves = np.array(ts[1:])
    g = oracle.replay_grad("robertson", wl["params"][:1], wl["y0"][:1], wl["t0"], wl["t1"], saves,
                           np.array([0, len(h)]), h)
    np.testing.assert_allclose(g["y_save"][0].sum(-1), 1.0, atol=1e-13)
