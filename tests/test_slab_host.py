"""Host protocol of the slab split with one slab per rank, as gloo ranks on the CPU.

Every event exchanges two messages with each neighbouring slab (Sec. 2.5's
ghost-layer refresh): a slab's upper-face buffer goes to the upper neighbour's
lower receive buffer and its lower-face buffer to the lower neighbour's upper
receive buffer.  The ranks here send buffers that name their sender and side
and check that each receive buffer holds the right neighbour's right face,
with periodic and reflective k axes, two and three ranks (two ranks on a
periodic axis are each other's neighbour on both sides), and one rank alone.
"""
import json
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _pattern(torch, rank, side, phase, n=64):
    return torch.arange(n, dtype=torch.int64) + 1000000 * (rank + 1) + 1000 * (side + 1) + 100 * phase


def _rank_main(rank, world, port, periodic, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist

    import paper_1605_03726_gb300 as psc

    dist.init_process_group("gloo", rank=rank, world_size=world)
    ex = psc.SlabRanks(rank, world, periodic)
    got = {}
    for phase in range(3):                      # claim and commit messages of consecutive events
        send = [_pattern(torch, rank, s, phase) for s in (0, 1)]
        recv = [torch.full((64,), -1, dtype=torch.int64) for _ in (0, 1)]
        ex.exchange(send, recv)
        got[phase] = [recv[0].tolist(), recv[1].tolist()]
    dist.barrier()
    dist.destroy_process_group()
    with open(os.path.join(out_dir, "r%d.json" % rank), "w") as f:
        json.dump({"nb": ex.nb, "got": got}, f)


@pytest.mark.parametrize("world,periodic", [(2, True), (3, True), (3, False), (2, False)])
def test_slab_exchange_routes_faces_to_neighbours(tmp_path, world, periodic):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp

    sys.path.insert(0, ROOT)
    import paper_1605_03726_gb300 as psc

    port = _free_port()
    mp.start_processes(_rank_main, args=(world, port, periodic, str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    for rank in range(world):
        r = json.load(open(tmp_path / ("r%d.json" % rank)))
        lo = psc.slab_neighbour(rank, world, 0, periodic)
        hi = psc.slab_neighbour(rank, world, 1, periodic)
        assert r["nb"] == [lo, hi]
        for phase in range(3):
            recv_lo, recv_hi = r["got"][str(phase)]
            # from below: the lower neighbour's upper face; from above: the upper neighbour's lower face
            if lo is None:
                assert recv_lo == [-1] * 64
            else:
                assert recv_lo == _pattern(torch, lo, 1, phase).tolist()
            if hi is None:
                assert recv_hi == [-1] * 64
            else:
                assert recv_hi == _pattern(torch, hi, 0, phase).tolist()


def test_single_rank_slab_is_its_own_neighbour_on_a_periodic_axis():
    torch = pytest.importorskip("torch")
    sys.path.insert(0, ROOT)
    import paper_1605_03726_gb300 as psc

    ex = psc.SlabRanks(0, 1, True)
    assert ex.nb == [0, 0]
    send = [_pattern(torch, 0, s, 0) for s in (0, 1)]
    recv = [torch.zeros(64, dtype=torch.int64) for _ in (0, 1)]
    ex.exchange(send, recv)
    assert torch.equal(recv[0], send[1]) and torch.equal(recv[1], send[0])
    wall = psc.SlabRanks(0, 1, False)
    assert wall.nb == [None, None]
    recv = [torch.zeros(64, dtype=torch.int64) for _ in (0, 1)]
    wall.exchange(send, recv)
    assert not recv[0].any() and not recv[1].any()
