"""Independent chains across processes (Sec. 3.4): the host-side bookkeeping
of the replica launch — disjoint chain ids, a barrier, and the max of the
ranks' times — on two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1402_1763_gb300 import replicas


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, lr = replicas.rank_world()
    base = replicas.chain_id_base(r, 16)
    replicas.barrier(dist)
    t = replicas.max_over_ranks(1.5 + r, dist)
    out[rank] = (r, w, lr, base, t)
    dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_max_time_and_disjoint_chains():
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
    assert out[0] == (0, 2, 0, 0, 2.5)
    assert out[1] == (1, 2, 1, 16, 2.5)


def test_single_process_defaults(monkeypatch):
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    assert replicas.rank_world() == (0, 1, 0)
    assert replicas.max_over_ranks(3.25, None) == 3.25
    replicas.barrier(None)
