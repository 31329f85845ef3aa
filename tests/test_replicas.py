"""Multi-GPU bench host logic on CPU: world-size-2 gloo ranks reduce their
timings with MAX and report all ranks' solves over the slowest rank's time."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_1901_00654_gb300 import replicas
    seconds = [2.0, 5.0][rank]                 # rank 1 is the slow one
    rate, worst = replicas.job_rate(3, seconds, world, "cpu")
    out[rank] = (rate, worst)
    dist.destroy_process_group()


def test_job_rate_two_gloo_ranks():
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    for r in (0, 1):
        rate, worst = res[r]
        assert worst == 5.0                    # max over ranks
        assert rate == pytest.approx(2 * 3 / 5.0)


def test_job_rate_single_process():
    from paper_1901_00654_gb300 import replicas
    assert replicas.job_rate(4, 2.0, 1) == (2.0, 2.0)
