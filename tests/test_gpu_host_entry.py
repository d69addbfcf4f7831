"""gs_solve_grad_host: host arrays in and out, the ensemble solved in chunks
with the copies overlapping the solves. Trajectories are independent, so every
per-trajectory result must equal gs_solve_grad's on the whole ensemble bit for
bit, whatever the chunking (ragged last chunk included) and whether the host
memory is page-locked or not."""
import numpy as np
import pytest
import torch

from paper_2609_02876_gb300 import api, build
from paper_2609_02876_gb300 import workloads as W
from tests.test_gpu_tsit5 import dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def host(x, pin):
    t = torch.from_numpy(np.ascontiguousarray(x))
    return t.pin_memory() if pin else t


@pytest.mark.parametrize("name,n,chunk,pin,method", [("lorenz", 5000, 1024, True, None),
                                                      ("lorenz", 3000, 0, False, None),
                                                      ("vdp", 2049, 512, True, "verner7"),
                                                      ("robertson", 700, 256, False, None)])
def test_host_entry_equals_device_entry_bit_for_bit(name, n, chunk, pin, method):
    wl = W.make(name, n)
    ref = api.solve_grad(name, dev(wl["params"].T), dev(wl["y0"].T), wl["t0"], wl["t1"], wl["save_t"], wl["rtol"],
                         wl["atol"], layout="soa", method=method)
    got = api.solve_grad_host(name, host(wl["params"].T, pin), host(wl["y0"].T, pin), wl["t0"], wl["t1"],
                              wl["save_t"], wl["rtol"], wl["atol"], chunk=chunk, method=method)
    for k in ("loss", "params_bar", "y0_bar", "status"):
        assert not got[k].is_cuda
        np.testing.assert_array_equal(got[k].numpy(), ref[k].cpu().numpy(), err_msg=k)


def test_host_entry_shared_weights_run_as_one_chunk():
    wl = W.make("nrob", 300)
    w32 = np.asarray(wl["w"], dtype=np.float32)
    SW = torch.as_tensor(w32, device="cuda")
    ref = api.solve_grad("nrob", dev(wl["params"].T), dev(wl["y0"].T), wl["t0"], wl["t1"], wl["save_t"], wl["rtol"],
                         wl["atol"], layout="soa", shared_w=SW)
    got = api.solve_grad_host("nrob", host(wl["params"].T, True), host(wl["y0"].T, True), wl["t0"], wl["t1"],
                              wl["save_t"], wl["rtol"], wl["atol"], shared_w=SW, chunk=64)
    np.testing.assert_array_equal(got["params_bar"].numpy(), ref["params_bar"].cpu().numpy())
    np.testing.assert_array_equal(got["shared_w_bar"].cpu().numpy(), ref["shared_w_bar"].cpu().numpy())
