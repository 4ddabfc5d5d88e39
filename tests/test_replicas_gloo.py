"""Multi-GPU runs are independent replicas (no data-path collective): each
rank advances its own chains from its own seed, and the whole-job rate is all
ranks' units over the slowest rank's time.  Checked with two gloo ranks on the
CPU; the oracle stands in for a rank's chains."""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, out):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        import bench
        import oracle
        # each rank's chains: a small 2D lattice advanced by the oracle
        oracle.build()
        model = oracle.Model(dim=2, L=(4, 4), beta=0.44)
        sums = oracle.run_chains(model, 2, oracle.FORM_FP64, bench.replica_seed(rank), eps=0.1,
                                 n_md=4, n=6)
        elapsed = 1.0 + rank          # rank 1 is the slow one
        rate, tmax = bench.job_rate(100, elapsed, ws)
        out[rank] = (rate, tmax, np.asarray(sums).ravel().tolist())
    finally:
        dist.destroy_process_group()


@pytest.mark.timeout(300)
def test_replicas_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        mp.start_processes(_rank, args=(2, _free_port(), out), nprocs=2, start_method="spawn")
        r0, r1 = out[0], out[1]
    assert r0[1] == r1[1] == 2.0                  # max over ranks
    assert r0[0] == r1[0] == pytest.approx(100 * 2 / 2.0)
    assert r0[2] != r1[2]                         # different seeds, different chains
