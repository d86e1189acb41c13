"""Multi-process host logic on CPU (world size 2, gloo): volume partitioning
(every volume to exactly one rank, balanced by voxels), max/sum over ranks as
used by the benchmark's timing, and the noise streams of sharded runs: the
Philox volume word (noise_id) is the volume's global index, so a rank that
draws the noise of its share of a batch gets exactly what one process drawing
the whole batch gets, and replicas (one batch per rank) draw distinct
streams.  The noise itself comes from the FP64 oracle, run in each rank."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_1811_11226_b300 import dist as D


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


NOISE_SEED, NOISE_GRID, NOISE_Q = 4242, (16, 12), np.arange(0, 16 * 12 * 8, 37)


def _noise(noise_id):
    from oracle import ref
    return ref.noise(NOISE_SEED, noise_id, *NOISE_GRID, NOISE_Q)


def _worker(rank, world, port, weights, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    r, w, _ = D.init_from_env("gloo")
    assert (r, w) == (rank, world)
    mine = D.partition(weights, world, rank)
    D.barrier()
    mx = D.reduce_max(float(rank + 1.5))
    sm = D.reduce_sum(float(sum(weights[i] for i in mine)))
    # noise of this rank's share of the batch (volume word = global index), and
    # of its first replica volume (volume word from replica_noise_ids)
    shard = {i: _noise(i) for i in mine}
    replica = _noise(D.replica_noise_ids(4, rank)[0])
    out[rank] = (mine, mx, sm, shard, replica)
    import torch.distributed as dist
    dist.destroy_process_group()


def test_partition_max_and_sum_over_two_gloo_ranks():
    rng = np.random.default_rng(0)
    weights = [int(v) for v in rng.integers(1, 100, 37)]
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.start_processes(_worker, args=(world, port, weights, out), nprocs=world,
                           start_method="spawn")
        res = dict(out)
    got = sorted(i for r in range(world) for i in res[r][0])
    assert got == list(range(len(weights)))
    assert all(res[r][1] == 2.5 for r in range(world))
    assert all(res[r][2] == sum(weights) for r in range(world))
    loads = [sum(weights[i] for i in res[r][0]) for r in range(world)]
    assert max(loads) - min(loads) <= max(weights)
    # sharded noise equals the noise one process draws for the same volumes
    for r in range(world):
        for i, z in res[r][3].items():
            assert np.array_equal(z, _noise(i)), (r, i)
    # replicas draw distinct streams
    assert not np.array_equal(res[0][4], res[1][4])


def test_replica_noise_ids_are_disjoint():
    ids = [set(D.replica_noise_ids(64, r)) for r in range(8)]
    assert all(len(s) == 64 for s in ids)
    assert len(set().union(*ids)) == 64 * 8


@pytest.mark.parametrize("world", [1, 2, 3, 7])
def test_partition_properties(world):
    rng = np.random.default_rng(world)
    weights = [int(v) for v in rng.integers(1, 50, 40)]
    parts = [D.partition(weights, world, r) for r in range(world)]
    flat = [i for p in parts for i in p]
    assert flat == list(range(len(weights)))
    total = sum(weights)
    for p in parts:
        assert abs(sum(weights[i] for i in p) - total / world) <= max(weights)


def test_single_process_helpers_are_identity():
    assert D.reduce_max(3.0) == 3.0 and D.reduce_sum(2.0) == 2.0
    D.barrier()
