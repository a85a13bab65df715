"""Multi-process host logic of the benchmark on CPU (gloo, world size 2): each
rank renders its own batch of poses (weak scaling, no data-path collective) and
the job time is the slowest rank's."""
import os
import socket
import statistics

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


def _timing_worker(rank, world, port, out):
    """One rank of a CPU stand-in job: the step sleeps 20 ms on rank 0 and 60 ms on
    rank 1, timed by the bench's own per-rank path and aggregated across ranks."""
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import time

    import bench
    per_rank = [bench.timed_steps(lambda: time.sleep(0.02 + 0.04 * rank), 3, clock="host")]
    ms, value = bench.job_timing(world, 640000, per_rank, dist)
    if rank == 0:
        out.put((ms, value, [statistics.mean(per_rank[0])]))
    else:
        out.put(("rank1", [statistics.mean(per_rank[0])]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_time_steps_and_report_the_job():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_timing_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    r0 = next(g for g in got if g[0] != "rank1")
    r1 = next(g for g in got if g[0] == "rank1")
    ms, value, own0 = r0
    own1 = r1[1]
    # the job time is the slowest rank's (rank 1 sleeps 60 ms per step)
    assert ms[0] == pytest.approx(max(own0[0], own1[0]))
    assert ms[0] >= 55.0
    # whole-job throughput: both ranks' rays over the slowest rank's time
    assert value[0] == pytest.approx(2 * 640000 / (ms[0] * 1e-3) / 1e9)


@pytest.mark.parametrize("env,gpus", [({}, 2), ({"WORLD_SIZE": "1"}, 2), ({"WORLD_SIZE": "4"}, 8), ({}, 0)])
def test_bench_refuses_a_gpu_count_it_was_not_launched_with(env, gpus):
    import bench
    with pytest.raises(SystemExit):
        bench.resolve_world(gpus, env)


def test_bench_world_from_torchrun_env():
    import bench
    assert bench.resolve_world(1, {}) == (0, 1, 0)
    assert bench.resolve_world(2, {"WORLD_SIZE": "2", "RANK": "1", "LOCAL_RANK": "1"}) == (1, 2, 1)


def test_bench_main_refuses_gpus_2_without_torchrun(monkeypatch):
    import bench
    monkeypatch.delenv("WORLD_SIZE", raising=False)
    monkeypatch.setattr("sys.argv", ["bench.py", "--gpus", "2", "--steps", "1", "--warmup", "3"])
    with pytest.raises(SystemExit) as e:
        bench.main()
    assert "torch.distributed.run" in str(e.value)


def test_job_throughput_counts_all_ranks():
    import bench
    assert bench.job_throughput(1, 640000, 1.0) == pytest.approx(0.64)
    assert bench.job_throughput(4, 640000, 2.0) == pytest.approx(1.28)
