"""The N > 1 path of the benchmark on CPU: two gloo ranks.

Ranks evaluate disjoint k1-slabs (no data-path collective: the k-points are independent),
the step time is the maximum over ranks, and the slab sums of all ranks add up to the
full-mesh sum (checked here with the oracle standing in for each rank's GPU work and one
SUM all-reduce standing in for the caller combining the ranks' results).
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist          # noqa: E402
import torch.multiprocessing as mp        # noqa: E402

import bench                              # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out_path):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import tbgen
    from oracle import kubo_oracle as O
    m = tbgen.random_tb(4, 1, 1.0, 2)
    kmesh = (4, 3, 2)
    plane = kmesh[1] * kmesh[2]
    n_slabs = kmesh[0]                    # one k1-plane per slab
    E_F = [-0.2, 0.3]
    S = np.zeros((1, len(E_F)))
    mine = []
    for step in range(n_slabs // world):
        s = bench.slab_of(rank, world, step, n_slabs)
        mine.append(s)
        S += O.ahc(m.H_R, m.R, kmesh, E_F, kidx=np.arange(s * plane, (s + 1) * plane))
    t = torch.from_numpy(S.copy())
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    slabs = [None] * world
    dist.all_gather_object(slabs, mine)
    slowest = bench.max_over_ranks(10.0 + rank, dist, "cpu")
    if rank == 0:
        full = O.ahc(m.H_R, m.R, kmesh, E_F)
        np.savez(out_path, total=t.numpy(), full=full, slowest=slowest,
                 slabs=np.array(slabs, dtype=object), allow_pickle=True)
    dist.destroy_process_group()


def test_two_gloo_ranks_partition_the_mesh_and_take_the_slowest_time(tmp_path):
    out = str(tmp_path / "res.npz")
    mp.start_processes(_rank_main, args=(2, _free_port(), out), nprocs=2, join=True,
                       start_method="spawn")
    r = np.load(out, allow_pickle=True)
    slabs = [list(x) for x in r["slabs"]]
    assert sorted(slabs[0] + slabs[1]) == [0, 1, 2, 3]        # disjoint, every slab once
    assert float(r["slowest"]) == 11.0
    assert np.max(np.abs(r["total"] - r["full"])) <= 1e-14 * np.max(np.abs(r["full"]))


@pytest.mark.parametrize("world", [1, 2, 4, 8])
def test_slabs_are_disjoint_within_a_step(world):
    n_slabs = 32
    for step in range(9):
        s = [bench.slab_of(r, world, step, n_slabs) for r in range(world)]
        assert len(set(s)) == world
