"""Multi-process host logic of the benchmark on CPU (gloo, world size 2): each
rank renders its own batch of poses (weak scaling, no data-path collective) and
the job time is the slowest rank's."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from paper_2208_12737_gb300 import inputs
    cfg = inputs.CT
    poses, g = bench.rank_batch(cfg, rank)
    t = torch.from_numpy(np.concatenate([poses.ravel(), g.ravel()[:64]]).astype(np.float64))
    gathered = [torch.zeros_like(t) for _ in range(world)]
    dist.all_gather(gathered, t)
    # per-rank timings: rank r is slower in the first entry, faster in the second
    mx = bench.max_over_ranks([1.0 + rank, 10.0 - rank], dist)
    if rank == 0:
        out.put((torch.stack(gathered).numpy(), mx))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_shard_poses_and_take_the_slowest_time():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    gathered, mx = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert mx == [2.0, 10.0]
    a, b = gathered
    assert not np.allclose(a, b)  # distinct problems per rank
    # rank 0's batch is the single-GPU workload's batch
    import bench
    from paper_2208_12737_gb300 import inputs
    p0, g0 = bench.rank_batch(inputs.CT, 0)
    np.testing.assert_array_equal(p0, inputs.random_poses(inputs.CT["batch"], seed=inputs.CT["pose_seed"]))
    np.testing.assert_allclose(a[: p0.size], p0.ravel().astype(np.float64))


def test_job_throughput_counts_all_ranks():
    import bench
    assert bench.job_throughput(1, 640000, 1.0) == pytest.approx(0.64)
    assert bench.job_throughput(4, 640000, 2.0) == pytest.approx(1.28)
