"""Host logic of the multi-GPU bench path on CPU ranks (gloo, world size 2).

The chains are independent Markov chains (one walker per task in the paper's
MPI runtime): every rank runs its own batch with its own seed, the bench's only
collective is the max-reduction of the timing, and the whole-job throughput
adds the ranks' proposals.  This runs the same helpers bench.py uses, with
two CPU processes and no GPU.  The bin driver's one exchange, the sum of each
bin's accumulators over the ranks, is checked against one process holding all
the chains.
"""
import os
import socket

import numpy as np
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


class _Merged:
    """One process holding the chains of several fake ensembles side by side,
    concatenated along the chain axis: what the ranks hold together."""

    def __init__(self, parts):
        self.parts = parts
        self.n_chains = sum(p.n_chains for p in parts)

    def model_of(self, c):
        return self.parts[0].model_of(0)

    def sweep(self, n, stats=False):
        for p in self.parts:
            p.sweep(n, stats)

    def _cat(self, name, *a):
        outs = [getattr(p, name)(*a) for p in self.parts]
        return tuple(np.concatenate([o[i] for o in outs]) for i in range(len(outs[0])))

    def measure(self):
        return self._cat("measure")

    def measure_tau(self, n_tau, phases):
        return self._cat("measure_tau", n_tau, phases)

    def measure_corr(self, classes, n_class):
        return self._cat("measure_corr", classes, n_class)


def _sim_rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_1704_00131_gb300.simulation import Simulation
    from tests.test_simulation_host import FakeEnsemble
    res = Simulation(FakeEnsemble(n_chains=3, seed=rank), n_bins=4, sweeps_per_bin=3, warmup=1, tau=(4, None),
                     corr=([None], [2]), distributed=True).run()
    out[rank] = ({k: np.asarray(v).tolist() for k, v in res.mean.items()},
                 {k: np.asarray(v).tolist() for k, v in res.error.items()}, res.mean_sign)
    dist.barrier()
    dist.destroy_process_group()


def test_simulation_bins_are_summed_over_ranks():
    """Two gloo ranks, each with its own three chains, give (on both ranks) the
    result of one process holding all six chains: the bins' sums over chains are
    added over the ranks once per bin."""
    from paper_1704_00131_gb300.simulation import Simulation
    from tests.test_simulation_host import FakeEnsemble
    port = _free_port()
    manager = mp.Manager()
    out = manager.dict()
    mp.spawn(_sim_rank, args=(2, port, out), nprocs=2, join=True)
    ref = Simulation(_Merged([FakeEnsemble(n_chains=3, seed=0), FakeEnsemble(n_chains=3, seed=1)]), n_bins=4,
                     sweeps_per_bin=3, warmup=1, tau=(4, None), corr=([None], [2])).run()
    for rank in (0, 1):
        mean, err, msign = out[rank]
        assert msign == pytest.approx(ref.mean_sign, rel=1e-12)
        assert set(mean) == set(ref.mean)
        for k in ref.mean:
            assert np.allclose(mean[k], ref.mean[k], rtol=1e-12, atol=1e-14), k
            assert np.allclose(err[k], ref.error[k], rtol=1e-10, atol=1e-14), k


def _failing_rank(rank, world, port, out):
    import datetime

    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=20))
    from paper_1704_00131_gb300.simulation import Simulation
    from tests.test_simulation_host import FakeEnsemble

    class Dies(FakeEnsemble):
        def sweep(self, n, stats=False):
            if self.counter >= 4:                       # the fifth sweep: inside the second bin
                raise RuntimeError("injected failure of this rank's chains")
            return super().sweep(n, stats)

    ens = Dies(n_chains=3, seed=rank) if rank == 1 else FakeEnsemble(n_chains=3, seed=rank)
    try:
        Simulation(ens, n_bins=4, sweeps_per_bin=3, corr=([None], [2]), distributed=True).run()
        out[rank] = "finished"
    except Exception as e:                              # noqa: BLE001 - the outcome is what the test checks
        out[rank] = type(e).__name__ + ": " + str(e)[:200]
    # rank 1 leaves between its own steps, with no collective in flight; rank 0 is
    # waiting in the bin's all-reduce and must get an error, not hang


def test_distributed_bins_report_a_lost_rank():
    """A rank whose chains fail leaves the run between steps; the other rank's
    next per-bin all-reduce ends with an error (peer gone, or the process group's
    20 s timeout) instead of waiting forever.  The failure is injected on the host."""
    import time
    port = _free_port()
    manager = mp.Manager()
    out = manager.dict()
    t0 = time.monotonic()
    mp.spawn(_failing_rank, args=(2, port, out), nprocs=2, join=True)
    assert out[1].startswith("RuntimeError: injected failure")
    assert out[0] != "finished"
    assert time.monotonic() - t0 < 120
