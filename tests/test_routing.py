"""Serving replicas: the routing rule (host-only C ABI), and one process per
GPU agreeing on every request's owner from all-gathered figures (two gloo
ranks on the CPU)."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as tmp

from paper_2011_03602_gb300 import oo


def test_route_pick_rule():
    # most free bytes among the replicas with room
    assert oo.oo_route_pick([10, 30, 20], [0, 5, 0], 15) == 1
    # a replica without room is skipped however empty it is
    assert oo.oo_route_pick([10, 30, 20], [0, 5, 0], 25) == 1
    assert oo.oo_route_pick([40, 30, 20], [9, 0, 0], 35) == 0
    # ties on free bytes: fewer in flight, then the lower index
    assert oo.oo_route_pick([30, 30, 30], [4, 2, 2], 1) == 1
    assert oo.oo_route_pick([30, 30], [0, 0], 1) == 0
    # nobody has room: fewest in flight (it queues there)
    assert oo.oo_route_pick([10, 5, 8], [3, 1, 2], 100) == 1
    with pytest.raises(ValueError):
        oo.oo_route_pick([], [], 1)


def test_route_batch_charges_each_decision():
    # 100 and 60 free: 50 -> 0 (50 left), 50 -> 1 (60 > 50), 50 -> 0 (50 vs 10)
    assert list(oo.oo_route_batch([100, 60], [0, 0], [50, 50, 50])) == [0, 1, 0]
    # equal replicas alternate
    assert list(oo.oo_route_batch([64, 64], [0, 0], [8, 8, 8, 8])) == [0, 1, 0, 1]
    # the batch is the same as picking one by one with the charges applied
    rng = np.random.default_rng(3)
    f = rng.integers(1 << 20, 1 << 30, 4).astype(np.uint64)
    q = rng.integers(0, 5, 4).astype(np.uint64)
    needs = rng.integers(1 << 10, 1 << 28, 50).astype(np.uint64)
    got = oo.oo_route_batch(f, q, needs)
    f2, q2 = f.astype(object), q.astype(object)
    for j, nd in enumerate(needs):
        r = oo.oo_route_pick(np.array(f2, np.uint64), np.array(q2, np.uint64), int(nd))
        assert got[j] == r
        f2[r] = max(0, int(f2[r]) - int(nd))
        q2[r] = int(q2[r]) + 1


def test_footprint_estimates():
    g = oo.serve_request("gemm", A=np.zeros((64, 100)), B=np.zeros((100, 32)), C=np.zeros((64, 32)),
                         prec=oo.OO_PREC_SPLIT3_BF16)
    assert oo.oo_serve_footprint(g) == 8 * (64 * 100 + 100 * 32 + 64 * 32)
    g2 = oo.serve_request("gemm", A=np.zeros((64, 100)), B=np.zeros((100, 32)), C=np.zeros((64, 32)))
    assert oo.oo_serve_footprint(g2) > oo.oo_serve_footprint(g)  # FP64-equivalent: plus digit slices
    f = oo.serve_request("fft", x=np.zeros(4096, complex), X=np.zeros(4096, complex))
    assert oo.oo_serve_footprint(f) == 32 * 4096
    j = oo.serve_request("jacobi", I=9, J=10, K=11, iters=1, p=np.zeros(990, np.float32), res=np.zeros(1))
    assert oo.oo_serve_footprint(j) >= 14 * 9 * 10 * 11 * 4


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, out):
    import torch
    import torch.distributed as dist
    from paper_2011_03602_gb300 import oo as oo_r
    from paper_2011_03602_gb300 import replicas
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # every rank generates the same request stream; figures differ per rank
        rng = np.random.default_rng(11)
        needs = rng.integers(1 << 20, 1 << 29, 40)
        free = [3 << 30, 2 << 30][rank]
        in_flight = [1, 0][rank]
        owners = replicas.route_round(needs, free, in_flight)
        gathered = [torch.zeros(len(needs), dtype=torch.int32) for _ in range(world)]
        dist.all_gather(gathered, torch.from_numpy(np.asarray(owners, np.int32)))
        out[rank] = (list(map(int, owners)), [list(map(int, g)) for g in gathered],
                     list(map(int, oo_r.oo_route_batch([3 << 30, 2 << 30], [1, 0], needs))))
    finally:
        dist.destroy_process_group()


def test_two_ranks_agree_on_every_owner():
    world, port = 2, _free_port()
    mgr = tmp.Manager()
    out = mgr.dict()
    tmp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
    o0, g0, ref = out[0]
    o1, g1, _ = out[1]
    assert o0 == o1 == ref            # the same owners on both ranks, by the library's rule
    assert g0 == g1 == [o0, o0]       # each rank saw the other's owners equal its own
    assert set(o0) == {0, 1}          # both replicas serve
