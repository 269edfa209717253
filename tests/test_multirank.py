"""The multi-rank logic of bench.py (one process per GPU under torchrun) on
CPU: two gloo ranks, problems partitioned with no data-path collective, the
step time reduced as the maximum and the work as the sum over ranks."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, ws, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        share = bench.rank_share(range(48), ws, rank)
        ms, total = bench.reduce_over_ranks(torch, torch.device("cpu"), 10.0 + rank, len(share))
        out[rank] = (share, ms, total)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_partition_and_reduce():
    ws, port = 2, _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.start_processes(_rank, args=(ws, port, out), nprocs=ws, start_method="spawn")
        res = dict(out)
    shares = [res[r][0] for r in range(ws)]
    assert sorted(shares[0] + shares[1]) == list(range(48))
    assert not set(shares[0]) & set(shares[1])
    for r in range(ws):
        assert res[r][1] == 11.0          # max of 10.0 and 11.0
        assert res[r][2] == 48            # sum of the shares


def test_single_process_reduce_is_identity():
    assert bench.reduce_over_ranks(torch, torch.device("cpu"), 3.5, 7) == (3.5, 7)
