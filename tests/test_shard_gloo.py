"""Multi-rank host path on CPU (gloo, world size 2): sharded gradients equal the
unsharded ones, and the shared-weight (LV UDE) gradient summed across ranks
equals the single-process sum. The compute stand-in is the CPU oracle."""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2609_02876_gb300 import shard


def test_shard_range_partitions():
    for n in (0, 1, 7, 1024, 1000003):
        for world in (1, 2, 3, 8):
            spans = [shard.shard_range(n, r, world) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(spans, spans[1:]))
            sizes = [hi - lo for lo, hi in spans]
            assert max(sizes) - min(sizes) <= 1


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    from paper_2609_02876_gb300 import workloads as W
    wl = W.make("lv_ude", 12)
    lo, hi = shard.shard_range(12, rank, world)
    rec = oracle.record("lv_ude", wl["params"][lo:hi], wl["y0"][lo:hi], wl["t0"], wl["t1"], wl["save_t"],
                        wl["rtol"], wl["atol"], w=wl["w"], nthreads=1)
    g = oracle.replay_grad("lv_ude", wl["params"][lo:hi], wl["y0"][lo:hi], wl["t0"], wl["t1"], wl["save_t"],
                           rec["offsets"], rec["h"], w=wl["w"], nthreads=1)
    wsum = shard.sum_shared_grad(g["w_bar"])
    tmax = shard.max_over_ranks(float(rank + 1))
    out[rank] = {"lo": lo, "hi": hi, "pbar": g["params_bar"], "wsum": wsum, "tmax": tmax}
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_gloo_shards_match_single_process():
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.start_processes(_worker, args=(world, _free_port(), out), nprocs=world, start_method="spawn")
        res = dict(out)
    import oracle
    from paper_2609_02876_gb300 import workloads as W
    wl = W.make("lv_ude", 12)
    rec = oracle.record("lv_ude", wl["params"], wl["y0"], wl["t0"], wl["t1"], wl["save_t"], wl["rtol"], wl["atol"],
                        w=wl["w"], nthreads=1)
    g = oracle.replay_grad("lv_ude", wl["params"], wl["y0"], wl["t0"], wl["t1"], wl["save_t"], rec["offsets"],
                           rec["h"], w=wl["w"], nthreads=1)
    pbar = np.concatenate([res[r]["pbar"] for r in range(world)])
    np.testing.assert_array_equal(pbar, g["params_bar"])
    # the two ranks hold bit-identical sums, equal to the single-process sum up to FP64 reassociation
    np.testing.assert_array_equal(res[0]["wsum"], res[1]["wsum"])
    np.testing.assert_allclose(res[0]["wsum"], g["w_bar"], rtol=1e-13, atol=1e-13 * np.abs(g["w_bar"]).max())
    assert res[0]["tmax"] == res[1]["tmax"] == 2.0
