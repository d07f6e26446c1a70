"""Sharding of images over ranks (replicas, no data-path collective): balanced
contiguous ranges, a 2-rank gloo run on CPU whose gathered result equals the
unsharded one, and host-side detection of a rank that never arrives."""
import datetime
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2607_10280_b300 import sharding, synth


def test_shard_ranges_tile_and_balance():
    rng = np.random.default_rng(0)
    sizes = synth.uneven_sizes(512)
    costs = [sharding.image_cost(int(p), 2, 16) for p in sizes]
    for world in (1, 2, 3, 4, 8):
        r = sharding.shard_ranges(costs, world)
        assert r[0][0] == 0 and r[-1][1] == len(costs)
        assert all(r[i][1] == r[i + 1][0] for i in range(world - 1))
        loads = [sum(costs[a:b]) for a, b in r]
        assert max(loads) <= sum(costs) / world + max(costs)      # within one image of ideal
    assert sum(b - a for a, b in sharding.shard_ranges([1.0] * 5, 8)) == 5   # more ranks than images
    costs = rng.random(37)
    assert sum(b - a for a, b in sharding.shard_ranges(costs, 4)) == 37


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, p, L, chi, out_path, fail_rank):
    import torch.distributed as dist
    from oracle import pipeline
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=20))
    X = synth.garment_pixels(6, p, seed=9)
    params = synth.circuit_params(L, p * p, seed=10)
    ranges = sharding.shard_ranges([sharding.image_cost(p, L, chi)] * len(X), world)
    a, b = ranges[rank]
    if rank == fail_rank:
        return                                   # this rank dies before the barrier
    local = np.stack([pipeline.pauli_cache(X[i], p, L, chi, "ladder", params) for i in range(a, b)]) \
        if b > a else np.zeros((0, 2 * p * (p - 1), 16))
    if fail_rank >= 0:
        try:
            dist.monitored_barrier(timeout=datetime.timedelta(seconds=3))
            np.save(out_path, np.array([0]))
        except RuntimeError as e:
            np.save(out_path, np.array([1 if str(fail_rank) in str(e) else 2]))
        return
    full = sharding.gather_to_root(local)
    if rank == 0:
        np.save(out_path, full)
    dist.destroy_process_group()


def test_two_rank_gather_equals_unsharded(tmp_path):
    from oracle import pipeline
    p, L, chi = 3, 2, 4
    out = str(tmp_path / "full.npy")
    mp.start_processes(_worker, args=(2, _free_port(), p, L, chi, out, -1), nprocs=2, start_method="spawn")
    got = np.load(out)
    X = synth.garment_pixels(6, p, seed=9)
    params = synth.circuit_params(L, p * p, seed=10)
    ref = np.stack([pipeline.pauli_cache(X[i], p, L, chi, "ladder", params) for i in range(len(X))])
    assert np.array_equal(got, ref)


def test_missing_rank_is_detected_on_the_host(tmp_path):
    out = str(tmp_path / "status.npy")
    mp.start_processes(_worker, args=(2, _free_port(), 3, 1, 2, out, 1), nprocs=2, start_method="spawn")
    assert int(np.load(out)[0]) == 1            # rank 0's barrier timed out naming rank 1
