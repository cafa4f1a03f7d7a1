"""Host logic of the multi-GPU bench path on CPU ranks (gloo, world size 2).

The chains are independent Markov chains (one walker per task in the paper's
MPI runtime): every rank runs its own batch with its own seed, the only
collective is the max-reduction of the timing, and the whole-job throughput
adds the ranks' proposals.  This runs the same helpers bench.py uses, with
two CPU processes and no GPU.
"""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, out):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from paper_1704_00131_gb300 import workloads as W
    seed = bench.rank_seed(rank)
    wl = W.config_c3(8)
    # a stand-in for the measured per-rank time: ranks differ
    ms = torch.tensor([100.0 + 50.0 * rank])
    t = bench.max_over_ranks(float(ms.item()), device="cpu")
    value = bench.whole_job_value(wl.proposals_per_sweep(), world, t)
    out[rank] = (seed, t, value)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks():
    import bench
    from paper_1704_00131_gb300 import workloads as W
    port = _free_port()
    manager = mp.Manager()
    out = manager.dict()
    mp.spawn(_rank_main, args=(2, port, out), nprocs=2, join=True)
    s0, t0, v0 = out[0]
    s1, t1, v1 = out[1]
    assert s0 != s1                      # independent chains per rank
    assert t0 == t1 == 150.0             # max over ranks
    props = W.config_c3(8).proposals_per_sweep()
    assert v0 == v1 == pytest.approx(2 * props / 0.150)
