"""Replica runs (bench.py --gpus N under torchrun): the host logic on two gloo ranks
on CPU.  Every rank runs its own chain; the job's time is its slowest rank's, the
throughput is every rank's units over that time, and the seeds differ by rank."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch.distributed as dist

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench

        # rank r measured 1 + r seconds for 3 units
        t = bench.max_over_ranks(1.0 + rank, world, "cpu")
        q.put((rank, t, bench.job_rate(3, world, t), bench.rank_seed(7, rank)))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_replicas_report_the_slowest_rank():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert [o[1] for o in out] == [2.0, 2.0]  # both ranks see the slowest time
    assert [o[2] for o in out] == [3.0, 3.0]  # 2 ranks x 3 units / 2 s
    assert out[0][3] != out[1][3]  # independent chains


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks(1.5, 1, "cpu") == 1.5
    assert bench.job_rate(4, 1, 2.0) == 2.0
    assert bench.rank_seed(7, 0) == 7


def test_reference_arm_runs_on_rank_zero_only(capsys):
    """Under torchrun the reference arm's other ranks exit without work or output."""
    sys.path.insert(0, ROOT)
    import bench

    class Args:
        steps, warmup, gpus = 1, 0, 2

    wl = bench.WORKLOADS[bench.DEFAULT_WORKLOAD]
    bench.run_reference(Args(), bench.DEFAULT_WORKLOAD, wl, rank=1, world=2)
    assert capsys.readouterr().out == ""


def test_reference_line_is_consistent_with_its_own_clock(capsys):
    """ms_per_step is the wall time of one bounded oracle sample, and value is the
    fraction of a trajectory that sample covers over that time."""
    sys.path.insert(0, ROOT)
    import json

    import bench

    class Args:
        steps, warmup, gpus = 2, 1, 1

    name = "hmc_fp64_L8_Nt40"
    bench.run_reference(Args(), name, bench.WORKLOADS[name], rank=0, world=1)
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    w = line["work_per_step"]
    assert line["impl"] == "reference" and line["unit"] == "traj/s"
    assert 0 < w["fraction_of_unit"] < 1
    assert abs(line["value"] - w["fraction_of_unit"] / (line["ms_per_step"] / 1e3)) <= 1e-9 * line["value"]
    assert abs(line["value"] * w["extrapolated_s_per_unit"] - 1.0) < 1e-12


if __name__ == "__main__":
    sys.exit(pytest.main([__file__, "-q"]))
