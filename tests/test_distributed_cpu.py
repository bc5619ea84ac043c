"""Multi-process host logic of the benchmark on the CPU (gloo, world size 2).

Each rank evaluates its contiguous i-range of one system with the oracle;
the gathered shards must equal the unsharded evaluation bit for bit, and the
control-plane reductions (max of per-rank times, whole-job aggregate) must
combine ranks correctly. No GPU is involved.
"""

import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, result_path):
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import bench
    import oracle
    from paper_astro_ph_0703100_gb300 import synth

    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    oracle.set_threads(1)
    r, w = bench.dist_init("gloo")
    assert (r, w) == (rank, world)
    n = 1001
    p = synth.plummer(n, 5)
    lo, hi = bench.shard_rows(n, rank, world)
    acc, _ = oracle.force(p, p, 1e-3, rows=np.arange(lo, hi), potential=False)
    shards = [None] * world
    dist.all_gather_object(shards, (lo, hi, acc))
    t_max = bench.reduce_max(1.0 + rank)
    rate = bench.aggregate_rate(100.0, world, t_max)
    bench.barrier()
    if rank == 0:
        full = np.concatenate([s[2] for s in sorted(shards, key=lambda s: s[0])])
        ref, _ = oracle.force(p, p, 1e-3, potential=False)
        ok = (np.array_equal(full, ref) and [s[:2] for s in sorted(shards, key=lambda s: s[0])] ==
              [bench.shard_rows(n, k, world) for k in range(world)] and t_max == float(world) and
              rate == 100.0 * world / world)
        with open(result_path, "w") as f:
            f.write("ok" if ok else "mismatch")
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_reduce(tmp_path):
    out = tmp_path / "result.txt"
    mp.start_processes(_worker, args=(2, _free_port(), str(out)), nprocs=2, join=True, start_method="spawn")
    assert out.read_text() == "ok"


def test_shard_rows_partition():
    import bench

    for n in (0, 1, 7, 1000, 131072):
        for world in (1, 2, 3, 8):
            ranges = [bench.shard_rows(n, r, world) for r in range(world)]
            assert ranges[0][0] == 0 and ranges[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(ranges, ranges[1:]))
            assert max(h - l for l, h in ranges) - min(h - l for l, h in ranges) <= 1
